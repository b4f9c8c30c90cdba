// Alpha-profile form of the persistent batch kernel: the same schedule as batch.cu, with the
// last stage's output (FAM pair FFT, SSCA row pass) reduced straight into each signal's
// alpha profile (largest |S|^power per alpha column) by atomic maxima on the float bits
// (non-negative floats order like their bit patterns), so the SCD itself is never written.
#include "batch_kernel.cuh"

namespace scd {
namespace bk {
namespace {
template <bool FAM, bool TC>
cudaError_t prepare_one(int smem, int* blocks_per_sm) {
  cudaError_t e = cudaFuncSetAttribute(k_batch<FAM, TC, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_batch<FAM, TC, true>, kThreads, smem);
}
}  // namespace

cudaError_t prepare_kernel_profile(bool fam, bool tc, int smem, int* blocks_per_sm) {
  if (fam) return tc ? prepare_one<true, true>(smem, blocks_per_sm) : prepare_one<true, false>(smem, blocks_per_sm);
  return tc ? prepare_one<false, true>(smem, blocks_per_sm) : prepare_one<false, false>(smem, blocks_per_sm);
}

cudaError_t launch_batch_profile(bool fam, bool tc, int grid, int smem, const BatchArgs& A, cudaStream_t st) {
  if (fam) {
    if (tc) k_batch<true, true, true><<<grid, kThreads, smem, st>>>(A);
    else k_batch<true, false, true><<<grid, kThreads, smem, st>>>(A);
  } else {
    if (tc) k_batch<false, true, true><<<grid, kThreads, smem, st>>>(A);
    else k_batch<false, false, true><<<grid, kThreads, smem, st>>>(A);
  }
  return cudaGetLastError();
}
}  // namespace bk
}  // namespace scd
