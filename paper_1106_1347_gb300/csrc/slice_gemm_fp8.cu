// The FP8-E4M3 instantiations of the persistent slice product, slice counts 1..10
// and tile widths 64 (up to 8 slices) and 32
// (one translation unit per format, so the build compiles them in parallel).
#include "slice_gemm.cuh"

namespace emu {

cudaError_t launch_slice_gemm_fp8(int s, int bn, unsigned grid, size_t smem, cudaStream_t st, const CUtensorMap &tmA,
                                  const CUtensorMap &tmB, const EmuParams &prm) {
    return dispatch_slice_gemm<true>(s, bn, grid, smem, st, tmA, tmB, prm);
}

cudaError_t launch_group_slice_gemm_fp8(int s, int bn, unsigned grid, size_t smem, cudaStream_t st, const EmuProblem *tab,
                                        const int64_t *begin, const GroupHeader *hdr) {
    return dispatch_group_slice_gemm<true>(s, bn, grid, smem, st, tab, begin, hdr);
}

cudaError_t slice_gemm_smem_attributes_fp8(int bytes) { return set_slice_gemm_smem<true>(bytes); }

}  // namespace emu
