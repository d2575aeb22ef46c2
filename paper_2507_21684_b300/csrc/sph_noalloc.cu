// Cell binning without allocation (sph_noalloc.h): cell keys, stable LSD radix sort and CSR
// cell ranges of one scene's particles, with every temporary in one statically sized device
// array.  The sort passes are the library's radix-sort kernels (sph_kernels.cu); the key and
// offset kernels here read plain FP32 positions instead of a scene's packed state.
#include <mutex>

#include "sph_noalloc.h"
#include "sph_runtime.h"

namespace sph {

DevSeg make_seg(const sph_params& p, int n_fluid, int cell_base, int p0, int p1, double max_abs_x);

namespace {

constexpr int kMaxN = SPH_NOALLOC_MAX_PARTICLES;
constexpr int kHistWords = 256 * 256;  // 256 digits x ceil(kMaxN / 2048) sort tiles
constexpr int kSumWords = 4096;        // block sums of the histogram scan (>= 2048 + 64)
constexpr size_t kWords = 3 * (size_t)kMaxN + kHistWords + kSumWords;
static_assert(4 * kWords == (size_t)SPH_NOALLOC_SCRATCH_BYTES, "scratch size and header disagree");
static_assert(256 * ((kMaxN + 2047) / 2048) <= kHistWords, "histogram scratch too small");

// The scratch: keys (two buffers) and one value buffer of the sort, histograms, scan sums.
static __device__ __align__(256) uint32_t g_scratch[kWords];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
uint32_t* g_ptr[kMaxDevices] = {};

// Device address of the scratch on the current device (looked up once per device).
uint32_t* scratch_ptr() {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_err("sph_cells_noalloc: device ordinal out of range");
    throw Fail{SPH_EINVAL};
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_ptr[dev]) {
    void* p = nullptr;
    CK(cudaGetSymbolAddress(&p, g_scratch));
    g_ptr[dev] = (uint32_t*)p;
  }
  return g_ptr[dev];
}

// Cell key of x_k in FP64: floor((x wrapped into the box - lo) / cell edge), clamped to the
// grid (the same decision a scene makes from its uploaded positions).
template <int D>
__global__ void k_keys_plain(DevSeg s, const float* __restrict__ x, int n, uint32_t* __restrict__ keys,
                             uint32_t* __restrict__ ids) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  int cc3[3] = {0, 0, 0};
#pragma unroll
  for (int q = 0; q < D; ++q) {
    const double xq = (double)x[(size_t)k * D + q];
    double xw = xq;
    if ((s.periodic_mask >> q) & 1) {
      const double f = floor(__ddiv_rn(__dsub_rn(xq, s.lo_d[q]), s.L_d[q]));
      xw = __dsub_rn(xq, __dmul_rn(s.L_d[q], f));
    }
    double c = floor(__ddiv_rn(__dsub_rn(xw, s.lo_d[q]), s.cs_d[q]));
    c = fmin(fmax(c, 0.0), (double)(s.n[q] - 1));
    cc3[q] = (int)c;
  }
  keys[k] = (uint32_t)((cc3[2] * s.n[1] + cc3[1]) * s.n[0] + cc3[0]);
  ids[k] = (uint32_t)k;
}

// cell_start[c] = first sorted position whose key is >= c, c = 0 .. C: thread k fills the
// cells in (key[k-1], key[k]] (key[-1] = -1, key[n] = C).
__global__ void k_offsets_plain(const uint32_t* __restrict__ keys, int n, int C, int32_t* __restrict__ start) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > n) return;
  const int lo = (k == 0) ? 0 : (int)keys[k - 1] + 1;
  const int hi = (k < n) ? (int)keys[k] : C;
  for (int c = lo; c <= hi; ++c) start[c] = k;
}

__global__ void k_fill_zero(int32_t* __restrict__ start, long long len) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < len) start[k] = 0;
}

__global__ void k_copy_ids(const uint32_t* __restrict__ src, int n, int32_t* __restrict__ dst) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) dst[k] = (int32_t)src[k];
}

void run(const sph_params& p, const float* x, int n, int32_t* start, int64_t start_len, int32_t* ids,
         int32_t* n_cells, cudaStream_t st) {
  if (n < 0 || n > kMaxN)
    einval("sph_cells_noalloc: n = " + std::to_string(n) + " outside [0, " + std::to_string(kMaxN) +
           "] (the size of the library's static scratch)");
  const DevSeg s = make_seg(p, n, 0, 0, n, 0.0);
  const long long C = (long long)s.n[0] * s.n[1] * s.n[2];
  if (n_cells) *n_cells = (int32_t)C;
  if (!start || start_len < C + 1)
    einval("sph_cells_noalloc: cell_start needs n_cells + 1 = " + std::to_string(C + 1) + " entries");
  if (n > 0 && (!x || !ids)) einval("sph_cells_noalloc: x and sorted_ids are required for n > 0");
  uint32_t* base = scratch_ptr();  // setup before anything is enqueued
  uint32_t* kA = base;
  uint32_t* kB = base + kMaxN;
  uint32_t* vA = base + 2 * (size_t)kMaxN;
  uint32_t* hist = base + 3 * (size_t)kMaxN;
  uint32_t* sums = hist + kHistWords;
  uint32_t* vB = reinterpret_cast<uint32_t*>(ids);  // the caller's output is the other value buffer
  if (n > 0) {
    const int nb = (n + 255) / 256;
    if (p.dim == 2)
      k_keys_plain<2><<<nb, 256, 0, st>>>(s, x, n, kA, vA);
    else
      k_keys_plain<3><<<nb, 256, 0, st>>>(s, x, n, kA, vA);
    CKL();
    int bits = 0;
    while ((1LL << bits) < C) ++bits;
    const int passes = std::max(1, (bits + 7) / 8);
    uint32_t *ki = kA, *vi = vA, *ko = kB, *vo = vB;
    const Arrays none{};
    for (int q = 0; q < passes; ++q) {
      if (p.dim == 2)
        launch_sort_pass<2>(ki, vi, ko, vo, n, 8 * q, hist, sums, nullptr, none, st);
      else
        launch_sort_pass<3>(ki, vi, ko, vo, n, 8 * q, hist, sums, nullptr, none, st);
      CKL();
      std::swap(ki, ko);
      std::swap(vi, vo);
    }
    if (vi != vB) {
      k_copy_ids<<<nb, 256, 0, st>>>(vi, n, ids);
      CKL();
    }
    k_offsets_plain<<<(n + 1 + 255) / 256, 256, 0, st>>>(ki, n, (int)C, start);
  } else {
    k_fill_zero<<<(unsigned)((C + 1 + 255) / 256), 256, 0, st>>>(start, C + 1);
  }
  CKL();
}

}  // namespace
}  // namespace sph

extern "C" int sph_cells_noalloc(const sph_params* params, const float* x, int32_t n, int32_t* cell_start,
                                 int64_t cell_start_len, int32_t* sorted_ids, int32_t* n_cells, void* stream) {
  if (!params) {
    sph::set_err("sph_cells_noalloc: NULL params");
    return SPH_EINVAL;
  }
  try {
    sph::run(*params, x, n, cell_start, cell_start_len, sorted_ids, n_cells, (cudaStream_t)stream);
  } catch (const sph::Fail& f) {
    return f.code;
  } catch (...) {
    sph::set_err("sph_cells_noalloc: unexpected internal exception");
    return SPH_EINTERNAL;
  }
  return SPH_OK;
}
