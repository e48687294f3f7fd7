"""Generate lcs_step.inc: one inline-PTX update of a W-word bit-vector per W.

The bit-parallel LCS step over a W x 64-bit vector V for one symbol with
match mask P (little-endian 32-bit halves v[0..2W), p[0..2W)) is

    u = V & P;   s = V + u  (one 64W-bit addition, carry out of the top dropped);
    V = s | (V & ~P)

The addition must be one unbroken add.cc / addc.cc chain, and the carry flag
is not preserved between separate asm statements, so the whole W-word update
is emitted as a single asm block per W.  lop3 with LUT 0xF4 computes
a | (b & ~c) for (a, b, c) = (s, V, P).

A slice of N words of a vector split across warps (LcsSlice<N>::run) takes
its carry in from the top bit of a mask register, shifting the mask left
(add.cc.u32 m, m, m), and appends its carry out at bit 0 of another
(addc.u32 o, o, o): sixteen steps in a row leave their carries in one
16-bit field, which the next slice reads back in the same order.

Run: python gen_lcs_step.py > lcs_step.inc   (the build does this when the
generated file is older than this script).
"""
import sys

MAX_W = 32


def emit(W: int) -> str:
    n = 2 * W
    lines = []
    lines.append("template <> __device__ __forceinline__ void lcs_step<%d>(uint32_t (&v)[%d], const uint32_t (&p)[%d]) {" % (W, n, n))
    body = ["{", ".reg .b32 u<%d>, s<%d>;" % (n, n)]
    for i in range(n):
        body.append("and.b32 u%d, %%%d, %%%d;" % (i, i, n + i))
    for i in range(n):
        if i == 0:
            op = "add.cc.u32" if n > 1 else "add.u32"
        elif i == n - 1:
            op = "addc.u32"
        else:
            op = "addc.cc.u32"
        body.append("%s s%d, %%%d, u%d;" % (op, i, i, i))
    for i in range(n):
        body.append("lop3.b32 %%%d, s%d, %%%d, %%%d, 0xF4;" % (i, i, i, n + i))
    body.append("}")
    asm = "\\n\\t".join(body)
    outs = ", ".join('"+r"(v[%d])' % i for i in range(n))
    ins = ", ".join('"r"(p[%d])' % i for i in range(n))
    lines.append('  asm("%s"\n      : %s\n      : %s);' % (asm, outs, ins))
    lines.append("}")
    return "\n".join(lines)


SLICE_MAX = 16


def emit_slice(N: int) -> str:
    n = 2 * N
    body = ["{", ".reg .b32 u<%d>, s<%d>;" % (n, n)]
    for i in range(n):
        body.append("and.b32 u%d, %%%d, %%%d;" % (i, i, n + 2 + i))
    body.append("add.cc.u32 %%%d, %%%d, %%%d;" % (n, n, n))  # CF = top bit of the carry-in mask
    for i in range(n):
        body.append("addc.cc.u32 s%d, %%%d, u%d;" % (i, i, i))
    body.append("addc.u32 %%%d, %%%d, %%%d;" % (n + 1, n + 1, n + 1))  # carry out into bit 0
    for i in range(n):
        body.append("lop3.b32 %%%d, s%d, %%%d, %%%d, 0xF4;" % (i, i, i, n + 2 + i))
    body.append("}")
    asm = "\\n\\t".join(body)
    outs = ", ".join(['"+r"(v[%d])' % i for i in range(n)] + ['"+r"(cin)', '"+r"(cout)'])
    ins = ", ".join('"r"(p[%d])' % i for i in range(n))
    return ("template <> struct LcsSlice<%d> {\n"
            "  __device__ __forceinline__ static void run(uint32_t (&v)[%d], const uint32_t (&p)[%d], "
            "uint32_t &cin, uint32_t &cout) {\n"
            '    asm("%s"\n        : %s\n        : %s);\n  }\n};' % (N, n, n, asm, outs, ins))


def main():
    out = ["// Generated by gen_lcs_step.py -- do not edit.",
           "// Bit-parallel LCS word update, one asm block per vector width W (64-bit words).",
           "template <int W> __device__ __forceinline__ void lcs_step(uint32_t (&v)[2 * W], const uint32_t (&p)[2 * W]);"]
    for W in range(1, MAX_W + 1):
        out.append(emit(W))
    out.append("// slices of up to %d words, carries in and out through bit masks" % SLICE_MAX)
    out.append("template <int N> struct LcsSlice;")
    for N in range(1, SLICE_MAX + 1):
        out.append(emit_slice(N))
    sys.stdout.write("\n".join(out) + "\n")


if __name__ == "__main__":
    main()
