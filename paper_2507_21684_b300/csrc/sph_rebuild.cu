// The cell-structure rebuild in one cooperative launch: cell keys -> stable LSD radix sort ->
// permute with cell ranges -> tile table -> list of wall tiles (App. B), with grid-wide barriers
// between the phases instead of kernel boundaries (device side in sph_rebuild_dev.cuh).
#include "sph_rebuild_dev.cuh"

namespace sph {

namespace {

template <int D>
__global__ void __launch_bounds__(kRbThreads) k_rebuild_coop(RebuildArgs r) {
  // the next kernel (the sweep, launched as a programmatic dependent) may be scheduled at once:
  // it waits for this grid's completion before its first memory access
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  if (r.flag && *(volatile const int*)r.flag == 0) return;  // no rebuild due: the whole grid leaves
  __shared__ RebuildSmem sm;
  rebuild_body<D>(r, sm);
}

}  // namespace

// CTAs per SM of the cooperative rebuild: more make a rebuild faster, fewer make the usual launch
// that finds no rebuild due (every step between rebuilds) cheaper.
#ifndef SPH_RB_CTAS_PER_SM
#define SPH_RB_CTAS_PER_SM 2
#endif

template <int D>
int rebuild_coop_grid() {
  int dev = 0, sms = 0, occ = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_rebuild_coop<D>, kRbThreads, 0) != cudaSuccess) return 0;
  return sms * std::min(occ, SPH_RB_CTAS_PER_SM);
}

template <int D>
cudaError_t launch_rebuild_coop(const RebuildArgs& r, int grid, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kRbThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_rebuild_coop<D>, r);
}

// Test hook of the bounded waits: a grid barrier that one CTA never reaches.
__global__ void k_debug_barrier(unsigned* bar, int* status) {
  if (blockIdx.x == 0) return;
  grid_barrier(bar, status);
}
cudaError_t launch_debug_barrier(unsigned* bar, int* status, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2);
  cfg.blockDim = dim3(32);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_debug_barrier, bar, status);
}

template int rebuild_coop_grid<2>();
template int rebuild_coop_grid<3>();
template cudaError_t launch_rebuild_coop<2>(const RebuildArgs&, int, cudaStream_t);
template cudaError_t launch_rebuild_coop<3>(const RebuildArgs&, int, cudaStream_t);

}  // namespace sph
