// Pixel kernel: one launch per pass of Fig. 1 (Algorithm
// AlbedoReWeightL1Filter) over every line of the plan; the per-CTA work is
// pixel_block (mf_pixel_body.cuh).
#include "mf_pixel_body.cuh"

namespace mf {

size_t pixel_smem_bytes(int B, int nj) { return pix_layout(B, 8 * nj).total + 128; }
int pixel_ctas_per_sm(int nj) { return pix_ctas_per_sm(nj); }

// One pass, one CTA per (row block, column tile).  The kernel is launched
// without the programmatic attribute (measured: a pixel pass whose CTAs were
// placed early, as the solve's CTAs left, ran 4 us slower per launch); it
// still signals its dependents after its (then no-op) wait, so that the next
// solve's CTAs start their copies as the pass's CTAs finish.
template <int NJ>
__global__ void __launch_bounds__(kPixThreads, pix_ctas_per_sm(NJ))
    pixel_kernel(const __grid_constant__ CUtensorMap map, Params p, int mode, int accumulate,
                 int pass) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bars[kPixBars];
  if (threadIdx.x == 0) pixel_bars_init(bars);
  __syncthreads();
  PixPhases ph{};
  pixel_block<NJ, false>(map, p, mode, accumulate, pass, blockIdx.x, smem_raw, bars, ph, [] {
    pdl_wait();
    pdl_trigger();
    return true;
  });
}

#define MF_NJ_CASES(X) X(1) X(2) X(4) X(6) X(8) X(9) X(10) X(12) X(16)

cudaError_t pixel_set_attributes(int nj, size_t smem) {
#define MF_CASE(NJ)                                                                    \
  case NJ:                                                                             \
    return cudaFuncSetAttribute(pixel_kernel<NJ>,                                      \
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  switch (nj) { MF_NJ_CASES(MF_CASE) }
#undef MF_CASE
  return cudaErrorInvalidValue;
}

void pixel_launch(int nj, int grid, size_t smem, cudaStream_t s, const CUtensorMap& map,
                  const Params& p, int mode, int accumulate, int pass) {
#define MF_CASE(NJ)                                                        \
  case NJ:                                                                 \
    launch_kernel(pixel_kernel<NJ>, grid, kPixThreads, smem, s, false, map, p, mode, accumulate, \
                  pass);                                                 \
    return;
  switch (nj) { MF_NJ_CASES(MF_CASE) }
#undef MF_CASE
}

}  // namespace mf
