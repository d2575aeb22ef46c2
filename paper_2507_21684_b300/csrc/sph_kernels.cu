// CUDA kernels of the WCSPH step (sm_103a).  One pass of the method is
//   cell keys -> stable LSD radix sort -> cell ranges -> permute  (neighbour search, App. B)
//   -> wall extrapolation -> density summation                     (Sec. 2.3, App. A.6)
//   -> fused sweep: continuity + delta diffusion, Tait pressure, viscosity, gravity,
//      kick-drift epilogue                                          (Sec. 2.3, Sec. 3.4)
// and the mirrored adjoint sweep of a step (Sec. 2.2, 3.3).
#include "sph_kernels.cuh"
#include "sph_sort.cuh"

namespace sph {

// ================================================================== neighbour search
// ---- stable LSD radix sort, 8-bit digits, 2048-key tiles (device parts in sph_sort.cuh) ----
template <int D, int KEYS_FROM_STATE>
__global__ void __launch_bounds__(kSortThreads) k_sort_hist(const uint32_t* __restrict__ keys, int N, int shift,
                                                            uint32_t* __restrict__ hist, int nblocks,
                                                            const DevSeg* __restrict__ segs, Arrays a,
                                                            uint32_t* __restrict__ kcache) {
  __shared__ uint32_t h[256];
  sort_hist_tile<D, KEYS_FROM_STATE>(blockIdx.x, keys, N, shift, hist, nblocks, segs, a, h, kcache);
}

// Exclusive scan of n uint32 in place, 2048 per block; block totals to sums.
__global__ void __launch_bounds__(1024) k_scan_blocks(uint32_t* __restrict__ a, int n, uint32_t* __restrict__ sums) {
  __shared__ uint32_t sh[2048];
  const int base = blockIdx.x * 2048;
  for (int k = threadIdx.x; k < 2048; k += 1024) sh[k] = (base + k < n) ? a[base + k] : 0u;
  __syncthreads();
  // Blelloch up-sweep / down-sweep
  for (int d = 1; d < 2048; d <<= 1) {
    int idx = (threadIdx.x + 1) * (d << 1) - 1;
    if (idx < 2048) sh[idx] += sh[idx - d];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (sums) sums[blockIdx.x] = sh[2047];
    sh[2047] = 0;
  }
  __syncthreads();
  for (int d = 1024; d >= 1; d >>= 1) {
    int idx = (threadIdx.x + 1) * (d << 1) - 1;
    if (idx < 2048) {
      uint32_t t = sh[idx - d];
      sh[idx - d] = sh[idx];
      sh[idx] += t;
    }
    __syncthreads();
  }
  for (int k = threadIdx.x; k < 2048; k += 1024)
    if (base + k < n) a[base + k] = sh[k];
}

// Exclusive scan of up to 16384 values in one CTA of 1024 threads (16 consecutive per thread).
__global__ void __launch_bounds__(1024) k_scan_single(uint32_t* __restrict__ a, int n) {
  __shared__ uint32_t wsum[32];
  const int t = threadIdx.x, base = t * 16;
  uint32_t v[16], run = 0;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    v[k] = (base + k < n) ? a[base + k] : 0u;
    const uint32_t x = v[k];
    v[k] = run;
    run += x;
  }
  // exclusive scan of the per-thread totals: warp shuffles, then the warp totals
  const int lane = t & 31, w = t >> 5;
  uint32_t incl = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) wsum[w] = incl;
  __syncthreads();
  if (w == 0) {
    uint32_t ws = wsum[lane], wi = ws;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, wi, o);
      if (lane >= o) wi += y;
    }
    wsum[lane] = wi - ws;
  }
  __syncthreads();
  const uint32_t off = wsum[w] + incl - run;
#pragma unroll
  for (int k = 0; k < 16; ++k)
    if (base + k < n) a[base + k] = v[k] + off;
}

__global__ void k_scan_add(uint32_t* __restrict__ a, int n, const uint32_t* __restrict__ sums) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] += sums[i / 2048];
}

template <int D, int KEYS_FROM_STATE>
__global__ void __launch_bounds__(kSortThreads) k_sort_scatter(const uint32_t* __restrict__ kin,
                                                               const uint32_t* __restrict__ vin,
                                                               uint32_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                               int N, int shift, const uint32_t* __restrict__ hist,
                                                               int nblocks, const DevSeg* __restrict__ segs, Arrays a,
                                                               const uint32_t* __restrict__ kcache) {
  __shared__ ScatterSmem sm;
  sort_scatter_tile<D, KEYS_FROM_STATE>(blockIdx.x, kin, vin, kout, vout, N, shift, hist, nblocks, segs, a, sm, kcache);
}

template <int D>
__global__ void k_permute(const DevSeg* __restrict__ segs, int N, const uint32_t* __restrict__ perm, Arrays in,
                          Arrays out, const uint32_t* __restrict__ keys, int C, int* __restrict__ off,
                          float4* __restrict__ xb, int* __restrict__ boff) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k <= N) permute_one<D>(k, segs, N, perm, in, out, keys, C, off, xb, boff);
}

// ================================================================== state in/out
template <int D>
__global__ void k_upload(const DevSeg* __restrict__ segs, int seg, int n, int nf, int p0, const float* __restrict__ x,
                         const float* __restrict__ v, const float* __restrict__ rho, const float* __restrict__ mass,
                         Arrays a) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const DevSeg& s = segs[seg];
  PD<D> r;
  Cold c;
  bool wall = k >= nf;
  for (int q = 0; q < 3; ++q) {
    c.hi[q] = (q < D) ? x[(size_t)k * D + q] : 0.f;
    c.lo[q] = 0.f;
    c.off[q] = 0.f;
  }
  c.rlo = 0.f;
  c.aux = 0.f;
  for (int q = 0; q < D; ++q) {
    r.x[q] = c.hi[q];
    r.v[q] = wall ? 0.f : v[(size_t)k * D + q];
  }
  r.rho = rho[k];
  r.m = wall ? -fabsf(mass[k]) : mass[k];
  r.p = tait_p(s, r.rho);
  r.V = mass[k] / r.rho;
  int j = p0 + k;
  store_pd<D>(a, j, r);
  store_cold<D>(a, j, c);
  a.meta[j] = make_uint2((uint32_t)k | (wall ? kWallBit : 0u), (uint32_t)seg);
}

template <int D>
__global__ void k_download(int N, Arrays a, const int* __restrict__ orig_base, float* __restrict__ x,
                           float* __restrict__ v, float* __restrict__ rho) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  uint2 m = a.meta[k];
  int o = (int)(m.x & ~kWallBit) + orig_base[m.y];
  PD<D> r = load_pd<D>(a, k);
  Cold c = load_cold<D>(a, k);
  for (int q = 0; q < D; ++q) {
    if (x) x[(size_t)o * D + q] = __fadd_rn(c.hi[q], c.lo[q]);
    if (v) v[(size_t)o * D + q] = r.v[q];
  }
  if (rho) rho[o] = __fadd_rn(r.rho, c.rlo);
}

// ================================================================== adjoint seeds and bookkeeping (Sec. 2.2)
// Adjoint state per particle (sorted order of the step): XB = (xbar, rhobar), VB = (vbar, -).
// Seeds for the pair terms: abar = dt (vbar' + dt xbar'), bbar = dt rhobar', and P' = dp/drho.
template <int D>
__global__ void k_adj_seed(const DevSeg* __restrict__ segs, int N, Arrays fw, const float4* __restrict__ XB,
                           const float4* __restrict__ VB, float4* __restrict__ S, float* __restrict__ Pp) {
  wait_prior_grid();
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");  // the next kernel of the adjoint step may launch
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const DevSeg& s = segs[fw.meta[k].y];
  PD<D> r = load_pd<D>(fw, k);
  float4 xb = XB[k], vb = VB[k];
  float xbs[3] = {xb.x, xb.y, xb.z}, vbs[3] = {vb.x, vb.y, vb.z}, ab[3];
  for (int q = 0; q < 3; ++q) ab[q] = (q < D) ? s.dt * fmaf(s.dt, xbs[q], vbs[q]) : 0.f;
  float bb = s.density_mode == 0 ? s.dt * xb.w : 0.f;  // drho is integrated in continuity mode only
  float pp = tait_slope(s, r.rho, r.p);
  if (D == 2) {
    S[k] = make_float4(ab[0], ab[1], bb, pp);
  } else {
    S[k] = make_float4(ab[0], ab[1], ab[2], bb);
    Pp[k] = pp;
  }
}


// Adjoint of the permutation of a rebuild: out[perm[k]] = in[k].
__global__ void k_adj_unpermute(int N, const uint32_t* __restrict__ perm, const float4* __restrict__ XBin,
                                const float4* __restrict__ VBin, float4* __restrict__ XBout, float4* __restrict__ VBout) {
  wait_prior_grid();
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");  // the next kernel of the adjoint step may launch
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  int d = (int)perm[k];
  XBout[d] = XBin[k];
  VBout[d] = VBin[k];
}

// adjoint state of the final step from original-order inputs: scatter into sorted order
template <int D>
__global__ void k_adj_load(int N, const uint2* __restrict__ meta, const int* __restrict__ orig_base,
                           const float* __restrict__ xb, const float* __restrict__ vb, const float* __restrict__ rb,
                           float4* __restrict__ XB, float4* __restrict__ VB) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  uint2 m = meta[k];
  int o = (int)(m.x & ~kWallBit) + orig_base[m.y];
  float a[3] = {0.f, 0.f, 0.f}, b[3] = {0.f, 0.f, 0.f};
  for (int q = 0; q < D; ++q) {
    if (xb) a[q] = xb[(size_t)o * D + q];
    if (vb) b[q] = vb[(size_t)o * D + q];
  }
  XB[k] = make_float4(a[0], a[1], a[2], rb ? rb[o] : 0.f);
  VB[k] = make_float4(b[0], b[1], b[2], 0.f);
}

// adjoint of the initial state, delivered in original order through the storage map
template <int D>
__global__ void k_adj_store(int N, const uint2* __restrict__ meta, const int* __restrict__ orig_base,
                            const float4* __restrict__ XB, const float4* __restrict__ VB, float* __restrict__ xb,
                            float* __restrict__ vb, float* __restrict__ rb) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  uint2 m = meta[k];
  int o = (int)(m.x & ~kWallBit) + orig_base[m.y];
  float4 a = XB[k], b = VB[k];
  float as[3] = {a.x, a.y, a.z}, bs[3] = {b.x, b.y, b.z};
  for (int q = 0; q < D; ++q) {
    if (xb) xb[(size_t)o * D + q] = as[q];
    if (vb) vb[(size_t)o * D + q] = bs[q];
  }
  if (rb) rb[o] = a.w;
}

// Copy a particle range of one scene between packed batches; the scene index of the
// destination is written into meta (the serving loop re-packs its active scenes).
template <int D>
__global__ void k_copy_range(Arrays src, int s0, Arrays dst, int d0, int n, int seg) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int i = s0 + k, j = d0 + k;
  dst.A[j] = src.A[i];
  dst.B[j] = src.B[i];
  dst.X[j] = src.X[i];
  dst.O[j] = src.O[i];
  if (D == 3) {
    dst.C[j] = src.C[i];
    dst.XL[j] = src.XL[i];
  }
  uint2 m = src.meta[i];
  m.y = (uint32_t)seg;
  dst.meta[j] = m;
}

// State of one scene (rows [p0, p0 + n) of a batch) in its original particle order.
template <int D>
__global__ void k_download_range(Arrays a, int p0, int n, float* __restrict__ x, float* __restrict__ v,
                                 float* __restrict__ rho) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int i = p0 + k;
  const int o = (int)(a.meta[i].x & ~kWallBit);
  PD<D> r = load_pd<D>(a, i);
  Cold c = load_cold<D>(a, i);
  for (int q = 0; q < D; ++q) {
    x[(size_t)o * D + q] = __fadd_rn(c.hi[q], c.lo[q]);
    v[(size_t)o * D + q] = r.v[q];
  }
  rho[o] = __fadd_rn(r.rho, c.rlo);
}

// ================================================================== launchers

// Exclusive scan of n uint32 values in place: one CTA up to 16384 values, else 2048 per block
// with the block totals in sums.
void launch_exclusive_scan(uint32_t* a, int n, uint32_t* sums, cudaStream_t st) {
  if (n <= 0) return;
  if (n <= 16384) {
    k_scan_single<<<1, 1024, 0, st>>>(a, n);
    return;
  }
  const int sb = (n + 2047) / 2048;
  k_scan_blocks<<<sb, 1024, 0, st>>>(a, n, sums);
  k_scan_blocks<<<1, 1024, 0, st>>>(sums, sb, nullptr);
  k_scan_add<<<(n + 255) / 256, 256, 0, st>>>(a, n, sums);
}

// One LSD pass.  With segs set, the keys of the current storage order are computed on the fly
// (first pass) and the values are the storage indices.
template <int D>
void launch_sort_pass(const uint32_t* kin, const uint32_t* vin, uint32_t* kout, uint32_t* vout, int N, int shift,
                      uint32_t* hist, uint32_t* sums, const DevSeg* segs, const Arrays& a, cudaStream_t st,
                      bool xbins) {
  if (N <= 0) return;
  int nb = (N + kSortTile - 1) / kSortTile;
  if (segs) {
    // the first pass computes the keys from the state once: the histogram launch stores them in
    // kin (which the first pass does not read otherwise) and the scatter launch reads them there
    uint32_t* kc = const_cast<uint32_t*>(kin);
    if (xbins && D == 3)
      k_sort_hist<D, 2><<<nb, kSortThreads, 0, st>>>(kin, N, shift, hist, nb, segs, a, kc);
    else
      k_sort_hist<D, 1><<<nb, kSortThreads, 0, st>>>(kin, N, shift, hist, nb, segs, a, kc);
    launch_exclusive_scan(hist, 256 * nb, sums, st);
    if (xbins && D == 3)
      k_sort_scatter<D, 2><<<nb, kSortThreads, 0, st>>>(kin, vin, kout, vout, N, shift, hist, nb, segs, a, kc);
    else
      k_sort_scatter<D, 1><<<nb, kSortThreads, 0, st>>>(kin, vin, kout, vout, N, shift, hist, nb, segs, a, kc);
  } else {
    k_sort_hist<D, 0><<<nb, kSortThreads, 0, st>>>(kin, N, shift, hist, nb, segs, a, nullptr);
    launch_exclusive_scan(hist, 256 * nb, sums, st);
    k_sort_scatter<D, 0><<<nb, kSortThreads, 0, st>>>(kin, vin, kout, vout, N, shift, hist, nb, segs, a, nullptr);
  }
}

int sort_scratch_words(int N) {
  int nb = (N + kSortTile - 1) / kSortTile;
  return 256 * nb + 2048 + 64;
}

template <int D>
void launch_permute(const DevSeg* segs, int N, const uint32_t* perm, const Arrays& in, const Arrays& out,
                    const uint32_t* keys, int C, int* off, float4* xb, cudaStream_t st, int* boff) {
  k_permute<D><<<(N + 1 + 255) / 256, 256, 0, st>>>(segs, N, perm, in, out, keys, C, off, xb, boff);
}

// Whole-state copy (every array of the records) in one launch.
template <int D>
__global__ void k_copy_state(int N, Arrays src, Arrays dst) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < N) copy_state_one<D>(k, src, dst);
}
template <int D>
void launch_copy_state(int N, const Arrays& src, const Arrays& dst, cudaStream_t st) {
  if (N > 0) k_copy_state<D><<<(N + 255) / 256, 256, 0, st>>>(N, src, dst);
}

// Rebuild decision of one step, taken on the device: rebuild when the cells have served
// `interval` sweeps or when some particle has moved farther than half the skin since the last
// build (maxr > 1, from the previous sweep).  Sets the graph's conditional and the counters.
__global__ void k_rebuild_decide(RebuildCtl* ctl, int interval, int count, cudaGraphConditionalHandle h) {
  const unsigned r = (ctl->since >= interval || __uint_as_float(ctl->maxr) > 1.f) ? 1u : 0u;
  cudaGraphSetConditional(h, r);
  ctl->since = r ? count : ctl->since + count;
  ctl->maxr = 0u;
  ctl->rebuilds += r;
  ctl->call_rebuilds += r;
}
void launch_rebuild_decide(RebuildCtl* ctl, int interval, int count, cudaGraphConditionalHandle h, cudaStream_t st) {
  k_rebuild_decide<<<1, 1, 0, st>>>(ctl, interval, count, h);
}
template <int D>
void launch_upload(const DevSeg* segs, int seg, int n, int nf, int p0, const float* x, const float* v, const float* rho,
                   const float* mass, const Arrays& a, cudaStream_t st) {
  if (n > 0) k_upload<D><<<(n + 255) / 256, 256, 0, st>>>(segs, seg, n, nf, p0, x, v, rho, mass, a);
}
template <int D>
void launch_download(int N, const Arrays& a, const int* orig_base, float* x, float* v, float* rho, cudaStream_t st) {
  if (N > 0) k_download<D><<<(N + 255) / 256, 256, 0, st>>>(N, a, orig_base, x, v, rho);
}
template <int D>
void launch_adj_seed(const DevSeg* segs, int N, const Arrays& fw, const float4* XB, const float4* VB, float4* S,
                     float* Pp, cudaStream_t st) {
  if (N > 0) {
    PdlLaunch L((N + 255) / 256, 256, 0, st);
    cudaLaunchKernelEx(&L.cfg, k_adj_seed<D>, segs, N, fw, XB, VB, S, Pp);
  }
}
void launch_adj_unpermute(int N, const uint32_t* perm, const float4* XBin, const float4* VBin, float4* XBout,
                          float4* VBout, cudaStream_t st) {
  if (N > 0) {
    PdlLaunch L((N + 255) / 256, 256, 0, st);
    cudaLaunchKernelEx(&L.cfg, k_adj_unpermute, N, perm, XBin, VBin, XBout, VBout);
  }
}
template <int D>
void launch_adj_load(int N, const uint2* meta, const int* orig_base, const float* xb, const float* vb, const float* rb,
                     float4* XB, float4* VB, cudaStream_t st) {
  if (N > 0) k_adj_load<D><<<(N + 255) / 256, 256, 0, st>>>(N, meta, orig_base, xb, vb, rb, XB, VB);
}
template <int D>
void launch_adj_store(int N, const uint2* meta, const int* orig_base, const float4* XB, const float4* VB, float* xb,
                      float* vb, float* rb, cudaStream_t st) {
  if (N > 0) k_adj_store<D><<<(N + 255) / 256, 256, 0, st>>>(N, meta, orig_base, XB, VB, xb, vb, rb);
}

template <int D>
void launch_copy_range(const Arrays& src, int s0, const Arrays& dst, int d0, int n, int seg, cudaStream_t st) {
  if (n > 0) k_copy_range<D><<<(n + 255) / 256, 256, 0, st>>>(src, s0, dst, d0, n, seg);
}
template <int D>
void launch_download_range(const Arrays& a, int p0, int n, float* x, float* v, float* rho, cudaStream_t st) {
  if (n > 0) k_download_range<D><<<(n + 255) / 256, 256, 0, st>>>(a, p0, n, x, v, rho);
}

#define SPH_INST_D(D)                                                                                          \
  template void launch_copy_range<D>(const Arrays&, int, const Arrays&, int, int, int, cudaStream_t);          \
  template void launch_download_range<D>(const Arrays&, int, int, float*, float*, float*, cudaStream_t);       \
  template void launch_permute<D>(const DevSeg*, int, const uint32_t*, const Arrays&, const Arrays&, const uint32_t*, \
                                  int, int*, float4*, cudaStream_t, int*);                                      \
  template void launch_copy_state<D>(int, const Arrays&, const Arrays&, cudaStream_t);                        \
  template void launch_sort_pass<D>(const uint32_t*, const uint32_t*, uint32_t*, uint32_t*, int, int, uint32_t*,   \
                                    uint32_t*, const DevSeg*, const Arrays&, cudaStream_t, bool);               \
  template void launch_upload<D>(const DevSeg*, int, int, int, int, const float*, const float*, const float*,   \
                                 const float*, const Arrays&, cudaStream_t);                                   \
  template void launch_download<D>(int, const Arrays&, const int*, float*, float*, float*, cudaStream_t);       \
  template void launch_adj_seed<D>(const DevSeg*, int, const Arrays&, const float4*, const float4*, float4*, float*, \
                                   cudaStream_t);                                                              \
  template void launch_adj_load<D>(int, const uint2*, const int*, const float*, const float*, const float*, float4*, \
                                   float4*, cudaStream_t);                                                     \
  template void launch_adj_store<D>(int, const uint2*, const int*, const float4*, const float4*, float*, float*, \
                                    float*, cudaStream_t);
SPH_INST_D(2)
SPH_INST_D(3)

}  // namespace sph
