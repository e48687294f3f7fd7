"""Generate lcs_step.inc: one inline-PTX update of a W-word bit-vector per W.

The bit-parallel LCS step over a W x 64-bit vector V for one symbol with
match mask P (little-endian 32-bit halves v[0..2W), p[0..2W)) is

    u = V & P;   s = V + u  (one 64W-bit addition, carry out of the top dropped);
    V = s | (V & ~P)

The addition must be one unbroken add.cc / addc.cc chain, and the carry flag
is not preserved between separate asm statements, so the whole W-word update
is emitted as a single asm block per W.  lop3 with LUT 0xF4 computes
a | (b & ~c) for (a, b, c) = (s, V, P).

For wide vectors the same step is also emitted in parts of up to 8 words
(LcsPart<N, MODE>::run<OFF, W>: words OFF/2 .. OFF/2 + N of a W-word
vector): the carry crosses from one part to the next through a register
(captured with addc.u32 c, 0, 0 and restored with add.cc.u32 t, c, 0xFFFFFFFF), so
only one part's Peq words need to be live at a time.  MODE 0 is the first
part (carry out), 1 a middle part (carry in and out), 2 the last (carry in).

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


PART_MAX = 8


def emit_part(N: int, mode: int) -> str:
    n = 2 * N
    body = ["{", ".reg .b32 u<%d>, s<%d>, t;" % (n, n)]
    for i in range(n):
        body.append("and.b32 u%d, %%%d, %%%d;" % (i, i, n + 1 + i))
    if mode != 0:
        body.append("add.cc.u32 t, %%%d, 0xFFFFFFFF;" % n)  # CF = carry in
    for i in range(n):
        if i == 0 and mode == 0:
            op = "add.cc.u32"
        elif i == n - 1 and mode == 2:
            op = "addc.u32"
        else:
            op = "addc.cc.u32"
        body.append("%s s%d, %%%d, u%d;" % (op, i, i, i))
    if mode != 2:
        body.append("addc.u32 %%%d, 0, 0;" % n)  # carry out
    for i in range(n):
        body.append("lop3.b32 %%%d, s%d, %%%d, %%%d, 0xF4;" % (i, i, i, n + 1 + i))
    body.append("}")
    asm = "\\n\\t".join(body)
    outs = ", ".join(['"+r"(v[OFF + %d])' % i for i in range(n)] + ['"+r"(c)'])
    ins = ", ".join('"r"(p[%d])' % i for i in range(n))
    return ("template <> struct LcsPart<%d, %d> {\n"
            "  template <int OFF, int W>\n"
            "  __device__ __forceinline__ static void run(uint32_t (&v)[2 * W], const uint32_t (&p)[%d], "
            "uint32_t &c) {\n"
            '    asm("%s"\n        : %s\n        : %s);\n  }\n};' % (N, mode, n, asm, outs, ins))


def main():
    out = ["// Generated by gen_lcs_step.py -- do not edit.",
           "// Bit-parallel LCS word update, one asm block per vector width W (64-bit words).",
           "template <int W> __device__ __forceinline__ void lcs_step(uint32_t (&v)[2 * W], const uint32_t (&p)[2 * W]);"]
    for W in range(1, MAX_W + 1):
        out.append(emit(W))
    out.append("// parts of up to %d words of a wide vector, the carry passed in c" % PART_MAX)
    out.append("template <int N, int MODE> struct LcsPart;")
    for N in range(1, PART_MAX + 1):
        for mode in (0, 1, 2):
            out.append(emit_part(N, mode))
    sys.stdout.write("\n".join(out) + "\n")


if __name__ == "__main__":
    main()
