"""Generate lcs_tpp_{a,b,c,d}.cu: the thread-per-pair LCS kernel instantiated
for every (W, R) the launch planner and the batch autotuner may pick
(W = 1..32 words, R in {1, 2, 4} rows per tile with R * W <= 32), split over
four translation units so they compile in parallel; and lcs_slice_{a,b}.cu:
the sliced kernel for every slice width WL = 1..16 words.

Run: python gen_lcs_tpp.py   (writes the four files next to this script)
"""
import os

HERE = os.path.dirname(os.path.abspath(__file__))
UNITS = {"a": range(1, 9), "b": range(9, 17), "c": range(17, 25), "d": range(25, 33)}


def rows_for(W):
    return [R for R in (1, 2, 4) if R * W <= 32]


def unit(name, widths):
    lines = ["// Generated by gen_lcs_tpp.py -- do not edit.",
             "// Thread-per-pair LCS kernels for row widths W = %d..%d (64-bit words)," % (widths[0], widths[-1]),
             "// R rows per tile.",
             '#include "lcs_kernels.cuh"', "", "namespace famsa {", "",
             "template <int W, int R>",
             "static cudaError_t go(const KParams &p, dim3 grid, cudaStream_t st) {",
             "  size_t smem = (size_t)R * W * kPeqWordU32 * sizeof(uint32_t);",
             "  k_lcs_tpp<W, R><<<grid, kTppThreads, smem, st>>>(p);",
             "  return cudaGetLastError();", "}", "",
             "cudaError_t launch_tpp_%s(int W, int R, const KParams &p, dim3 grid, cudaStream_t st) {" % name,
             "  switch (W * 8 + R) {"]
    for W in widths:
        for R in rows_for(W):
            lines.append("    case %d: return go<%d, %d>(p, grid, st);" % (W * 8 + R, W, R))
    lines += ["    default: return cudaErrorInvalidValue;", "  }", "}", "", "}  // namespace famsa", ""]
    return "\n".join(lines)


SLICE_UNITS = {"a": range(1, 9), "b": range(9, 17)}


def slice_unit(name, widths):
    lines = ["// Generated by gen_lcs_tpp.py -- do not edit.",
             "// Sliced LCS kernels for slice widths WL = %d..%d (64-bit words per warp)." % (widths[0], widths[-1]),
             '#include "lcs_kernels.cuh"', "", "namespace famsa {", "",
             "template <int WL>",
             "static cudaError_t go(int G, const KParams &p, dim3 grid, cudaStream_t st) {",
             "  const size_t smem = slice_smem(WL, G);",
             "  // the cap is per kernel: the largest any launch of it needs (16 slices),",
             "  // so that launches from other threads never lower it under this one",
             "  const size_t smem_max = slice_smem(WL, kSliceMaxG);",
             "  if (smem_max > 48 * 1024) {",
             "    cudaError_t e = cudaFuncSetAttribute(k_lcs_slice<WL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);",
             "    if (e != cudaSuccess) return e;",
             "  }",
             "  k_lcs_slice<WL><<<grid, 32 * G, smem, st>>>(p);",
             "  return cudaGetLastError();", "}", "",
             "cudaError_t launch_slice_%s(int WL, int G, const KParams &p, dim3 grid, cudaStream_t st) {" % name,
             "  switch (WL) {"]
    for W in widths:
        lines.append("    case %d: return go<%d>(G, p, grid, st);" % (W, W))
    lines += ["    default: return cudaErrorInvalidValue;", "  }", "}", "", "}  // namespace famsa", ""]
    return "\n".join(lines)


def main():
    for name, ws in UNITS.items():
        with open(os.path.join(HERE, "lcs_tpp_%s.cu" % name), "w") as f:
            f.write(unit(name, list(ws)))
    for name, ws in SLICE_UNITS.items():
        with open(os.path.join(HERE, "lcs_slice_%s.cu" % name), "w") as f:
            f.write(slice_unit(name, list(ws)))


if __name__ == "__main__":
    main()
