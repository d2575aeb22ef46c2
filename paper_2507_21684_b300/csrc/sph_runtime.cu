// Host runtime of the B300 WCSPH library: scene state in HBM, the per-step launch sequence,
// CUDA-graph replay of step chunks, gradient checkpointing and the reverse pass, and the
// extern "C" entry points declared in include/sph.h.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "sph.h"
#include "sph_runtime.h"
#include "sph_rebuild.cuh"

// Captured steps of 3D scenes with a Verlet skin rebuild in a conditional graph node whose body is
// the stand-alone rebuild (0) or in one cooperative launch (1).  On the 128^3 vortex with a 0.1 H
// skin: 1.185 against 1.213 ms per step (the cooperative rebuild of 2.1 M particles, with two CTAs
// per SM, takes 0.35 ms against 0.22 ms for the stand-alone kernels; a step's node costs about
// 10 us against 5 us for a cooperative launch that finds no rebuild due).  ncu profiles no kernel
// node of a graph with conditional nodes, so captures of 3D steps with a skin use the variant with
// the cooperative launch (the same kernels).
#ifndef SPH_COOP3
#define SPH_COOP3 0
#endif

namespace sph {

// ---------------------------------------------------------------- errors
static thread_local std::string g_err;
void set_err(const std::string& s) { g_err = s; }
const char* last_error() { return g_err.c_str(); }
void einval(const std::string& s) {
  set_err(s);
  throw Fail{SPH_EINVAL};
}

// ---------------------------------------------------------------- allocator
static sph_alloc_fn g_alloc = nullptr;
static sph_free_fn g_free = nullptr;
static void* g_alloc_ctx = nullptr;
static std::mutex g_alloc_mu;

void set_allocator(sph_alloc_fn a, sph_free_fn f, void* ctx) {
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  g_alloc = a;
  g_free = f;
  g_alloc_ctx = ctx;
}
void init_mem(DeviceMem& m) {
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  m.afn = g_alloc;
  m.ffn = g_free;
  m.actx = g_alloc_ctx;
  m.fctx = g_alloc_ctx;
}

DeviceMem::~DeviceMem() { release(); }
void* DeviceMem::get(size_t bytes) {
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~size_t(255);
  void* p = nullptr;
  if (afn) {
    p = afn(bytes, (void*)stream, actx);
    if (!p) {
      set_err("allocator hook returned NULL for " + std::to_string(bytes) + " bytes");
      throw Fail{SPH_ENOMEM};
    }
  } else {
    // stream-ordered pool allocation: cheap once the pool has grown (scenes of the serving loop
    // are created and destroyed at a high rate)
    static std::once_flag pool_once;
    std::call_once(pool_once, [] {
      int dev = 0;
      cudaMemPool_t pool;
      if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t keep = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
      }
    });
    cudaError_t e = cudaMallocAsync(&p, bytes, stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_err(std::string("cudaMallocAsync(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
      throw Fail{SPH_ENOMEM};
    }
  }
  blocks.push_back({p, bytes});
  total += bytes;
  return p;
}
void DeviceMem::release() {
  for (auto& b : blocks) {
    if (ffn)
      ffn(b.first, b.second, (void*)stream, fctx);
    else
      cudaFreeAsync(b.first, stream);
  }
  blocks.clear();
  total = 0;
}

// ---------------------------------------------------------------- kernel constants
static double kernel_cd(int dim, int kern) {
  const double pi = 3.14159265358979323846;
  if (kern == 0) return dim == 2 ? 9.0 / pi : 495.0 / (32.0 * pi);
  return dim == 2 ? 7.0 / pi : 21.0 / (2.0 * pi);
}

// Per-scene device parameters from the ABI parameters.
DevSeg make_seg(const sph_params& p, int n_fluid, int cell_base, int p0, int p1, double max_abs_x) {
  DevSeg s;
  std::memset(&s, 0, sizeof(s));
  if (p.dim != 2 && p.dim != 3) einval("dim must be 2 or 3");
  if (p.kernel != 0 && p.kernel != 1) einval("kernel must be SPH_KERNEL_WENDLAND4 or SPH_KERNEL_WENDLAND2");
  if (p.density_mode != 0 && p.density_mode != 1) einval("density_mode must be 0 or 1");
  if (p.diffusion != 0 && p.diffusion != 1) einval("diffusion must be SPH_DIFFUSION_MC or SPH_DIFFUSION_RENORM");
  if (!(p.shift >= 0.f) || !std::isfinite(p.shift)) einval("shift must be finite and >= 0");
  if (p.boundary != 0 && p.boundary != 1) einval("boundary must be SPH_BOUNDARY_SHEPARD or SPH_BOUNDARY_MDBC");
  if (!(p.H > 0.f) || !(p.dt > 0.f) || !(p.rho0 > 0.f) || !(p.c0 > 0.f) || !(p.gamma > 0.f))
    einval("H, dt, rho0, c0 and gamma must be positive");
  if (!(p.nu >= 0.f) || !(p.eps > 0.f) || !(p.skin >= 0.f) || p.rebuild_interval < 1)
    einval("nu >= 0, eps > 0, skin >= 0 and rebuild_interval >= 1 are required");
  s.dim = p.dim;
  s.kernel = p.kernel;
  s.density_mode = p.density_mode;
  s.periodic_mask = p.periodic_mask & ((1 << p.dim) - 1);
  double cmin = (double)p.H + (double)p.skin;
  long long ncell = 1;
  for (int k = 0; k < 3; ++k) {
    if (k < p.dim) {
      double L = p.box_hi[k] - p.box_lo[k];
      if (!(L > 0.0)) einval("box_hi must exceed box_lo on every axis");
      int n = (int)std::floor(L / cmin);
      if (n < 1) n = 1;
      if (((s.periodic_mask >> k) & 1) && n < 3) einval("a periodic axis needs at least 3 cells of edge >= H + skin");
      s.n[k] = n;
      s.L_d[k] = L;
      s.lo_d[k] = p.box_lo[k];
      s.cs_d[k] = L / n;
      s.L[k] = (float)L;
      s.lo[k] = (float)p.box_lo[k];
      s.invL[k] = (float)(1.0 / L);
    } else {
      s.n[k] = 1;
      s.L_d[k] = 1.0;
      s.cs_d[k] = 1.0;
      s.L[k] = 1.f;
      s.invL[k] = 1.f;
    }
    ncell *= s.n[k];
  }
  if (ncell > (1LL << 30)) einval("too many cells");
  if ((long long)s.n[1] * s.n[2] >= (1LL << 20)) einval("too many cell lines (ny * nz must be < 2^20)");
  s.cell_base = cell_base;
  s.p0 = p0;
  s.p1 = p1;
  s.nf = n_fluid;
  const int d = p.dim;
  const double H = p.H;
  s.H = p.H;
  s.H2 = (float)(H * H);
  s.H2_d = H * H;
  s.invH = (float)(1.0 / H);
  s.dt = p.dt;
  s.rho0 = p.rho0;
  s.c0 = p.c0;
  s.gamma = p.gamma;
  s.B = (float)((double)p.rho0 * p.c0 * p.c0 / p.gamma);
  s.nu = p.nu;
  s.shiftC = (float)((double)p.shift * (double)p.H * (double)p.H);
  s.dCv_dnu = (float)(2.0 * (d + 2) * p.rho0);
  s.Cv = (float)(2.0 * (d + 2) * p.rho0 * (double)p.nu);
  // h = H/2: the smoothing length of the delta-SPH diffusion and of the regulariser
  s.Cdel = p.density_mode == 0 ? (float)((double)p.delta * (0.5 * H) * p.c0) : 0.f;
  s.eH2 = (float)((double)p.eps * (0.5 * H) * (0.5 * H));
  double Cd = kernel_cd(d, p.kernel);
  s.Kw = (float)(Cd / std::pow(H, d));
  s.Kg = (float)((p.kernel == 0 ? -56.0 / 3.0 : -20.0) * Cd / std::pow(H, d + 2));
  s.Kh = (float)((p.kernel == 0 ? 560.0 : 60.0) * Cd / std::pow(H, d + 4));
  for (int k = 0; k < 3; ++k) s.g[k] = k < d ? p.g[k] : 0.f;
  // FP32 error of r^2 on folded positions is below ~8 ulp(|x|max) * |r|: guard band in r^2.
  // Only the box enters (folded positions stay within it up to one step of drift), so every
  // parameter of a scene, and with it the order of its sums, is fixed by sph_params alone.
  (void)max_abs_x;
  double box_abs = 1.0;
  for (int k = 0; k < p.dim; ++k) box_abs = std::max(box_abs, std::max(std::fabs(p.box_lo[k]), std::fabs(p.box_hi[k])));
  double ex = 8.0 * std::ldexp(box_abs, -23);
  double band = std::max(1e-5, 4.0 * ex / H);
  s.band_lo = (float)(H * H * (1.0 - band));
  s.band_hi = (float)(H * H * (1.0 + band));
  // cells farther than this from a target (at build time, in the folded frame) hold no
  // neighbour: H widened by the guard band, half the Verlet skin and FP32 rounding of the faces
  double Lmax = 1.0;
  for (int k = 0; k < p.dim; ++k) Lmax = std::max(Lmax, std::fabs(p.box_lo[k]) + s.L_d[k]);
  double reach = (H * (1.0 + 2.0 * band) + 0.5 * (double)p.skin) * (1.0 + 1e-5) + 16.0 * std::ldexp(Lmax, -23);
  s.trimR2 = (float)(reach * reach);
  for (int k = 0; k < 3; ++k) {
    s.cs[k] = (float)s.cs_d[k];
    s.invcs[k] = (float)(1.0 / s.cs_d[k]);
  }
  return s;
}

// Device bytes of the fused wall + sweep launch's task lists for one scene with walls, as
// Scene::alloc_all sizes them (the wall-tile index list and the two plan lists), for admission.
size_t wall_plan_bytes(const sph_params& p, int n_fluid, int n) {
  const DevSeg g = make_seg(p, n_fluid, 0, 0, n, 16.0);
  const long long C = (long long)g.n[0] * g.n[1] * g.n[2];
  const long long lines = (long long)g.n[1] * g.n[2];
  const int TP = p.dim == 2 ? TileCfg<2>::TP : TileCfg<3>::TP;
  const bool balanced = p.dim == 2 ? TileCfg<2>::CUT : TileCfg<3>::CUT;
  const long long upper = 3 * (((long long)n + TP - 1) / TP) + (C + TP - 1) / TP + 2 * lines + 1;
  const long long lu = balanced ? ((long long)n + TP - 1) / TP + (C + TP - 1) / TP + lines + 1 : upper;
  const long long u4 = p.dim == 2 ? TilePlan<2>::U4 : TilePlan<3>::U4;
  return (size_t)(2 * 16 * u4 * std::min(lu, upper) + 4 * upper + 8);
}

static int key_bits(long long C) {
  int b = 0;
  while ((1LL << b) < C) ++b;
  return b;
}

// ---------------------------------------------------------------- scene
// The caller's stream orders the scene's work.  Stream capture is not allowed on the legacy
// default stream, so a scene bound to stream 0 runs on a private non-blocking stream and
// joins the legacy stream with events at every entry point (enter) and before returning
// device outputs (leave).
void Scene::bind_stream(cudaStream_t user) {
  user_st = user;
  if (user == nullptr) {
    CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    own_stream = true;
    CK(cudaEventCreateWithFlags(&ev_in, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&ev_out, cudaEventDisableTiming));
  } else {
    st = user;
  }
  mem.stream = st;
}
void Scene::enter() {
  if (!own_stream) return;
  CK(cudaEventRecord(ev_in, nullptr));
  CK(cudaStreamWaitEvent(st, ev_in, 0));
}
void Scene::leave() {
  if (!own_stream) return;
  CK(cudaEventRecord(ev_out, st));
  CK(cudaStreamWaitEvent(nullptr, ev_out, 0));
}

Scene::~Scene() {
  if (st) cudaStreamSynchronize(st);
  for (auto& kv : graphs) cudaGraphExecDestroy(kv.second);
  for (auto& kv : adj_graphs) cudaGraphExecDestroy(kv.second.first);
  for (auto g : graph_templates) cudaGraphDestroy(g);
  for (auto e : event_pool) cudaEventDestroy(e);
  for (auto& e : prof_events) {
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  mem.release();
  if (own_stream) {
    cudaEventDestroy(ev_in);
    cudaEventDestroy(ev_out);
    cudaStreamDestroy(st);
  }
  if (st_body) cudaStreamDestroy(st_body);
  if (st_rep) cudaStreamDestroy(st_rep);
  for (int b = 0; b < 2; ++b) {
    if (ev_rep[b]) cudaEventDestroy(ev_rep[b]);
    if (ev_free[b]) cudaEventDestroy(ev_free[b]);
  }
}

void Scene::alloc_arrays(Arrays& a) {
  a.A = (float4*)mem.get(sizeof(float4) * N);
  a.B = (float4*)mem.get(sizeof(float4) * N);
  a.X = (float4*)mem.get(sizeof(float4) * N);
  a.O = (float4*)mem.get(sizeof(float4) * N);
  a.meta = (uint2*)mem.get(sizeof(uint2) * N);
  if (D == 3) {
    a.C = (float2*)mem.get(sizeof(float2) * N);
    a.XL = (float4*)mem.get(sizeof(float4) * N);
  } else {
    a.C = nullptr;
    a.XL = nullptr;
  }
}

void Scene::copy_arrays(const Arrays& dst, const Arrays& src) {
  CK(cudaMemcpyAsync(dst.A, src.A, sizeof(float4) * N, cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(dst.B, src.B, sizeof(float4) * N, cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(dst.X, src.X, sizeof(float4) * N, cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(dst.O, src.O, sizeof(float4) * N, cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(dst.meta, src.meta, sizeof(uint2) * N, cudaMemcpyDeviceToDevice, st));
  if (D == 3) {
    CK(cudaMemcpyAsync(dst.C, src.C, sizeof(float2) * N, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(dst.XL, src.XL, sizeof(float4) * N, cudaMemcpyDeviceToDevice, st));
  }
}

void Scene::setup_checked(const std::vector<sph_params>& prms, const std::vector<int>& nfs,
                          const std::vector<int>& nws, const std::vector<double>& max_abs_x) {
  S = (int)prms.size();
  D = prms[0].dim;
  kern = prms[0].kernel;
  summation = prms[0].density_mode == 1;
  renorm = !summation && prms[0].diffusion == 1;
  shifting = prms[0].shift > 0.f;
  mdbc = false;
  any_walls = false;
  skin = 0.f;  // the largest of the scenes' skins
  interval = prms[0].rebuild_interval;
  N = 0;
  C_tot = 0;
  segs.clear();
  orig_base.clear();
  for (int s = 0; s < S; ++s) {
    const sph_params& p = prms[s];
    if (p.dim != D || p.kernel != kern || (p.density_mode == 1) != summation)
      einval("all scenes of a batch must share dim, kernel and density mode");
    if (p.diffusion != prms[0].diffusion) einval("all scenes of a batch must share the diffusion form");
    if ((p.shift > 0.f) != (prms[0].shift > 0.f)) einval("all scenes of a batch must agree on particle shifting");
    if (p.boundary != prms[0].boundary) einval("all scenes of a batch must share the wall treatment");
    int n = nfs[s] + nws[s];
    if (nfs[s] < 0 || nws[s] < 0 || n < 1) einval("particle counts must be non-negative with at least one particle");
    if ((long long)N + n >= (1LL << 30)) einval("too many particles");
    DevSeg g = make_seg(p, nfs[s], C_tot, N, N + n, max_abs_x[s]);
    long long c = (long long)g.n[0] * g.n[1] * g.n[2];
    if ((long long)C_tot + c >= (1LL << 31)) einval("too many cells in total");
    segs.push_back(g);
    orig_base.push_back(N);
    N += n;
    C_tot += (int)c;
    if (nws[s] > 0) any_walls = true;
    if (nws[s] > 0 && p.boundary == 1) mdbc = true;
    if ((p.skin > 0.f) != (prms[0].skin > 0.f) || p.rebuild_interval != interval)
      einval("all scenes of a batch must share rebuild_interval, and either all or none have a Verlet skin");
    skin = std::max(skin, p.skin);
  }
  if (S >= 4096) einval("at most 4095 scenes per batch");
  static std::once_flag cfg_once;
  static cudaError_t cfg_err = cudaSuccess;
  std::call_once(cfg_once, [] { cfg_err = configure_passes(); });
  CK(cfg_err);
  nf_total = 0;
  for (int s = 0; s < S; ++s) nf_total += nfs[s];
  line_base_h.assign(S, 0);
  n_lines = 0;
  for (int s = 0; s < S; ++s) {
    line_base_h[s] = n_lines;
    n_lines += segs[s].n[1] * segs[s].n[2];
  }
  // lines are cut into chunks of TP cells and each chunk into ceil(count / TP) tiles: at most
  // N / TP + C_tot / TP + n_lines tiles (the bound below keeps a margin over that)
  {
    const int TP = D == 2 ? TileCfg<2>::TP : TileCfg<3>::TP;
    tiles_upper = 3 * ((N + TP - 1) / TP) + (C_tot + TP - 1) / TP + 2 * n_lines + 1;
  }
  bits = key_bits(C_tot);
  passes = std::max(1, (bits + 7) / 8);
  // Verlet skin: rebuild only when a particle has moved farther than skin/2 since the last
  // build (cells of edge >= H + skin then still hold every neighbour) or after `interval`
  // sweeps.  The threshold keeps 8 FP32 ulps of the largest coordinate in hand.
  {
    double Lmax = 1.0;
    for (int s = 0; s < S; ++s)
      for (int k = 0; k < D; ++k)
        Lmax = std::max(Lmax, std::max(std::fabs(segs[s].lo_d[k]), std::fabs(segs[s].lo_d[k] + segs[s].L_d[k])));
    // per scene: its own skin sets its displacement scale (a batch rebuilds all its scenes when
    // one of them has moved too far)
    dev_policy = skin > 0.f;
    inv_r2 = 0.f;
    for (int s = 0; s < S; ++s) {
      const double half = 0.5 * (double)prms[s].skin - 8.0 * std::ldexp(Lmax, -23);
      if (!(half > 0.0)) dev_policy = false;
    }
    for (int s = 0; s < S; ++s) {
      const double half = 0.5 * (double)prms[s].skin - 8.0 * std::ldexp(Lmax, -23);
      segs[s].inv_half2 = dev_policy ? (float)(1.0 / (half * half)) : 0.f;
      inv_r2 = std::max(inv_r2, segs[s].inv_half2);
    }
    // the adjoint's forward replay first tries a rebuild every 16 steps (every step without a skin)
    replay_k = dev_policy ? 16 : 1;
  }
  // the decision is taken by the sweep and the rebuild is one cooperative launch when the
  // device supports it (2D; 3D with SPH_COOP3); otherwise a one-thread kernel decides and a
  // conditional graph node rebuilds
  coop_grid = D == 2 ? rebuild_coop_grid<2>() : rebuild_coop_grid<3>();
  int coop_attr = 0, dev = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&coop_attr, cudaDevAttrCooperativeLaunch, dev));
  use_coop = dev_policy && coop_grid > 0 && coop_attr != 0 && (D == 2 || SPH_COOP3);
  // keys with x sub-bins for the warp-per-tile sweep; they need kXShift more key bits
  xorder = D == 3 && warp_sweep(D, N) && (long long)C_tot * kXBins < (1LL << 31);
  if (xorder) {
    bits = key_bits((long long)C_tot * kXBins);
    passes = std::max(1, (bits + 7) / 8);
  }
  if (N > 16384 * 2048) einval("too many particles for the radix sort scratch (max 33554432)");
}

void Scene::alloc_all() {
  dseg = (DevSeg*)mem.get(sizeof(DevSeg) * S);
  d_orig_base = (int*)mem.get(sizeof(int) * S);
  CK(cudaMemcpyAsync(dseg, segs.data(), sizeof(DevSeg) * S, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d_orig_base, orig_base.data(), sizeof(int) * S, cudaMemcpyHostToDevice, st));
  alloc_arrays(buf[0]);
  alloc_arrays(buf[1]);
  cur = 0;
  kA = (uint32_t*)mem.get(4 * (size_t)N);
  vA = (uint32_t*)mem.get(4 * (size_t)N);
  kB = (uint32_t*)mem.get(4 * (size_t)N);
  vB = (uint32_t*)mem.get(4 * (size_t)N);
  keys_sorted = kA;
  perm = vA;
  cell_off = (int*)mem.get(sizeof(int) * ((size_t)C_tot + 1));
  if (xorder) bin_off = (int*)mem.get(sizeof(int) * ((size_t)C_tot * kXBins + 1));
  scratch = (uint32_t*)mem.get(4 * (size_t)sort_scratch_words(N));
  line_base = (int*)mem.get(sizeof(int) * S);
  CK(cudaMemcpyAsync(line_base, line_base_h.data(), sizeof(int) * S, cudaMemcpyHostToDevice, st));
  tiles = (Tile*)mem.get(sizeof(Tile) * (size_t)tiles_upper);
  if (any_walls) {
    wall_tiles = (int*)mem.get(sizeof(int) * (size_t)tiles_upper);
    // a plan per listed tile: the lists hold at most the tiles of the table, which balanced cuts
    // bound by N / TP + cells / TP + lines
    const int TPd = D == 2 ? TileCfg<2>::TP : TileCfg<3>::TP;
    const bool balanced = D == 2 ? TileCfg<2>::CUT : TileCfg<3>::CUT;
    const long long lu = balanced ? (long long)(N + TPd - 1) / TPd + (C_tot + TPd - 1) / TPd + n_lines + 1
                                  : (long long)tiles_upper;
    const size_t pw = (size_t)(D == 2 ? TilePlan<2>::U4 : TilePlan<3>::U4) * (size_t)std::min<long long>(lu, tiles_upper);
    wall_plans = (uint4*)mem.get(sizeof(uint4) * pw);
    fluid_plans = (uint4*)mem.get(sizeof(uint4) * pw);
    d_nwall = (int*)mem.get(sizeof(int) * 2);
  }
  if (renorm) gradrho = (float4*)mem.get(sizeof(float4) * N);  // before any step is captured
  if (mdbc) {
    ghosts = (float4*)mem.get(sizeof(float4) * N);
    CK(cudaMemsetAsync(ghosts, 0, sizeof(float4) * N, st));
  }
  d_ntiles = (int*)mem.get(sizeof(int) * 2);
  d_tile_ctr = (int*)mem.get(sizeof(int) * 4);
  CK(cudaMemsetAsync(d_tile_ctr, 0, sizeof(int) * 4, st));  // tiled kernels leave it zeroed
  d_status = (int*)mem.get(sizeof(int) * (4 + (size_t)S));  // [0] error bits, [4 + s] scene s unstable
  d_pairs = (unsigned long long*)mem.get(sizeof(unsigned long long) * 2);
  d_ctl = (RebuildCtl*)mem.get(sizeof(RebuildCtl));
  CK(cudaMemsetAsync(d_ctl, 0, sizeof(RebuildCtl), st));
  d_bar = (unsigned*)mem.get(sizeof(unsigned) * 2);
  CK(cudaMemsetAsync(d_bar, 0, sizeof(unsigned) * 2, st));
  xbuild = (float4*)mem.get(sizeof(float4) * (size_t)N);
  if (D == 3) pairs_pos = (float*)mem.get(sizeof(float) * packed_pairs_floats(N));
  d_nubar = (double*)mem.get(sizeof(double) * (size_t)(S + 1));
  {
    long long mx = 1;
    for (const DevSeg& g : segs) mx = std::max(mx, (long long)(g.p1 - g.p0));
    sum_nch = sum_segments_chunks(mx);
    sum_chunk = (double*)mem.get(sizeof(double) * (size_t)S * sum_nch);
    sum_ctr = (int*)mem.get(sizeof(int) * (size_t)S);
    CK(cudaMemsetAsync(sum_ctr, 0, sizeof(int) * (size_t)S, st));  // left zeroed by the sums
  }
  CK(cudaMemsetAsync(d_status, 0, sizeof(int) * (4 + (size_t)S), st));
  CK(cudaMemsetAsync(d_pairs, 0, sizeof(unsigned long long) * 2, st));
  cells_valid = false;
  steps_since_build = 0;
}

void Scene::upload(int s, const float* x, const float* v, const float* rho, const float* mass, int is_dev) {
  const DevSeg& g = segs[s];
  int n = g.p1 - g.p0;
  const float *dx = x, *dv = v, *dr = rho, *dm = mass;
  float* staging = nullptr;
  if (!is_dev) {
    size_t nb = sizeof(float) * ((size_t)n * D * 2 + 2 * (size_t)n);
    staging = (float*)mem_tmp(nb);
    float* p = staging;
    CK(cudaMemcpyAsync(p, x, sizeof(float) * n * D, cudaMemcpyHostToDevice, st));
    dx = p;
    p += (size_t)n * D;
    if (v) CK(cudaMemcpyAsync(p, v, sizeof(float) * n * D, cudaMemcpyHostToDevice, st));
    else CK(cudaMemsetAsync(p, 0, sizeof(float) * n * D, st));
    dv = p;
    p += (size_t)n * D;
    CK(cudaMemcpyAsync(p, rho, sizeof(float) * n, cudaMemcpyHostToDevice, st));
    dr = p;
    p += n;
    CK(cudaMemcpyAsync(p, mass, sizeof(float) * n, cudaMemcpyHostToDevice, st));
    dm = p;
  } else if (!v) {
    float* p = (float*)mem_tmp(sizeof(float) * (size_t)n * D);
    CK(cudaMemsetAsync(p, 0, sizeof(float) * n * D, st));
    dv = p;
  }
  if (D == 2)
    launch_upload<2>(dseg, s, n, g.nf, g.p0, dx, dv, dr, dm, buf[cur], st);
  else
    launch_upload<3>(dseg, s, n, g.nf, g.p0, dx, dv, dr, dm, buf[cur], st);
  CKL();
  cells_valid = false;
}

void* Scene::mem_tmp(size_t bytes) {
  if (bytes > tmp_bytes) {
    tmp = mem.get(bytes);
    tmp_bytes = bytes;
  }
  return tmp;
}

TravArgs Scene::trav(const Arrays& a, const uint32_t* keys, const int* off, const int* boff) const {
  TravArgs t{};
  t.bin_off = boff;
  t.kshift = xorder ? kXShift : 0;  // every rebuild of such a scene writes keys with x sub-bins
  t.segs = dseg;
  t.N = N;
  t.a = a;
  t.keys = keys;
  t.cell_off = off;
  t.status = d_status;
  t.pair_count = d_pairs;
  t.tile_ctr = d_tile_ctr;
  t.packed = pairs_pos;
  return t;
}

cudaEvent_t Scene::take_event() {
  if (!event_pool.empty()) {
    cudaEvent_t e = event_pool.back();
    event_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  CK(cudaEventCreate(&e));
  return e;
}

// Kernel timing: CUDA events on the scene's stream around each timed launch.  Under stream
// capture the records become event-record nodes of the graph; every replay re-points them
// at fresh events (cudaGraphExecEventRecordNodeSetEvent), so each launch is timed.
void Scene::prof_begin(int cls) {
  if (!profiling || in_body) return;
  ProfEvent e;
  e.cls = cls;
  e.a = take_event();
  e.b = take_event();
  if (capturing) {
    CK(cudaEventRecordWithFlags(e.a, st, cudaEventRecordExternal));
    capture_events.push_back(e);
  } else {
    CK(cudaEventRecord(e.a, st));
    prof_events.push_back(e);
  }
}
void Scene::prof_end() {
  if (!profiling || in_body) return;
  if (capturing)
    CK(cudaEventRecordWithFlags(capture_events.back().b, st, cudaEventRecordExternal));
  else
    CK(cudaEventRecord(prof_events.back().b, st));
}

// Rebuild: stable sort of the current order by cell key (the first pass computes the keys) ->
// permute `in` into `out` and write the cell offsets to off_out -> tile table.  Returns the
// sorted keys and the permutation (in kA/kB, vA/vB unless copied to the given tape buffers).
std::pair<uint32_t*, uint32_t*> Scene::rebuild(const Arrays& in, const Arrays& out, uint32_t* keys_out,
                                               uint32_t* perm_out, int* off_out, Tile* tiles_out,
                                               int* ntiles_out, int* boff_out) {
  prof_begin(1);
  uint32_t *ki = kA, *vi = vA, *ko = kB, *vo = vB;
  uint32_t* hist = scratch;
  uint32_t* sums = scratch + (sort_scratch_words(N) - 2048 - 64);
  // boff_out (3D warp-per-tile sweep): keys with x sub-bins, so every cell comes out ordered by
  // sub-bin, and the sub-bins' offsets beside the cells'
  const bool bins = boff_out && D == 3;
  // the folded positions as the displacement check's reference: with a Verlet skin only
  float4* xref = dev_policy ? xbuild : nullptr;
  for (int p = 0; p < passes; ++p) {
    if (D == 2)
      launch_sort_pass<2>(ki, vi, ko, vo, N, 8 * p, hist, sums, p == 0 ? dseg : nullptr, in, st);
    else
      launch_sort_pass<3>(ki, vi, ko, vo, N, 8 * p, hist, sums, p == 0 ? dseg : nullptr, in, st, bins);
    CKL();
    std::swap(ki, ko);
    std::swap(vi, vo);
  }
  uint32_t* ks = ki;
  uint32_t* pm = vi;
  if (keys_out) {
    CK(cudaMemcpyAsync(keys_out, ks, 4 * (size_t)N, cudaMemcpyDeviceToDevice, st));
    ks = keys_out;
  }
  if (perm_out) {
    CK(cudaMemcpyAsync(perm_out, pm, 4 * (size_t)N, cudaMemcpyDeviceToDevice, st));
    pm = perm_out;
  }
  if (D == 2)
    launch_permute<2>(dseg, N, pm, in, out, ks, C_tot, off_out, xref, st);
  else
    launch_permute<3>(dseg, N, pm, in, out, ks, C_tot, off_out, xref, st, bins ? boff_out : nullptr);
  CKL();
  build_tiles(off_out, out.meta, tiles_out ? tiles_out : tiles, ntiles_out ? ntiles_out : d_ntiles);
  prof_end();
  const int scan_launches = 256 * ((N + 2047) / 2048) <= 16384 ? 1 : 3;
  launches += passes * (2 + scan_launches) + 1;
  return {ks, pm};
}

// Tile table of a cell structure (CSR offsets `off`), and the list of tiles holding wall
// particles (from the sorted meta words) when the scene has walls.
void Scene::build_tiles(const int* off, const uint2* meta, Tile* tl, int* ntl) {
  if (D == 2)
    launch_tiles<2>(dseg, S, line_base, n_lines, off, tl, ntl, st);
  else
    launch_tiles<3>(dseg, S, line_base, n_lines, off, tl, ntl, st);
  CKL();
  ++launches;
  if (any_walls && meta) {
    if (D == 2)
      launch_wall_tiles<2>(tl, ntl, tiles_upper, meta, wall_tiles, wall_plans, fluid_plans, d_nwall, st);
    else
      launch_wall_tiles<3>(tl, ntl, tiles_upper, meta, wall_tiles, wall_plans, fluid_plans, d_nwall, st);
    CKL();
    ++launches;
  }
}

// mDBC ghost nodes of the walls (n_wall rows per scene, in batch order) into the per-row table.
void Scene::set_ghosts(const float* g, int is_dev) {
  if (!mdbc) einval("sph_set_ghosts: the scene has no walls with boundary = SPH_BOUNDARY_MDBC");
  std::vector<float> h;
  size_t nw_total = 0;
  for (int s = 0; s < S; ++s) nw_total += (size_t)(segs[s].p1 - segs[s].p0 - segs[s].nf);
  const size_t n = nw_total * D;
  if (is_dev) {
    h.resize(n);
    CK(cudaMemcpyAsync(h.data(), g, sizeof(float) * n, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    g = h.data();
  }
  std::vector<float4> rows((size_t)N, make_float4(0.f, 0.f, 0.f, 0.f));
  size_t w = 0;
  for (int s = 0; s < S; ++s) {
    const int nw = segs[s].p1 - segs[s].p0 - segs[s].nf;
    for (int k = 0; k < nw; ++k, ++w) {
      float v[3] = {0.f, 0.f, 0.f};
      for (int q = 0; q < D; ++q) v[q] = g[w * D + q];
      if (!(std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]))) einval("sph_set_ghosts: non-finite ghost node");
      rows[(size_t)orig_base[s] + segs[s].nf + k] = make_float4(v[0], v[1], v[2], 0.f);
    }
  }
  CK(cudaMemcpyAsync(ghosts, rows.data(), sizeof(float4) * N, cudaMemcpyHostToDevice, st));
  CK(cudaStreamSynchronize(st));
  ghosts_set = true;
}

void Scene::need_ghosts() const {
  if (mdbc && !ghosts_set) einval("boundary = SPH_BOUNDARY_MDBC needs the walls' ghost nodes (sph_set_ghosts)");
}

void Scene::walls_pass(const TravArgs& t, const Tile* tl) {
  if (mdbc) {
    prof_begin(2);
    if (D == 2) {
      if (kern == 0) launch_mdbc<2, 0>(t, tl, wall_tiles, d_nwall, tiles_upper, ghosts, d_orig_base, st);
      else launch_mdbc<2, 1>(t, tl, wall_tiles, d_nwall, tiles_upper, ghosts, d_orig_base, st);
    } else {
      if (kern == 0) launch_mdbc<3, 0>(t, tl, wall_tiles, d_nwall, tiles_upper, ghosts, d_orig_base, st);
      else launch_mdbc<3, 1>(t, tl, wall_tiles, d_nwall, tiles_upper, ghosts, d_orig_base, st);
    }
    CKL();
    prof_end();
    ++launches;
    return;
  }
  prof_begin(2);
  if (D == 2) {
    if (kern == 0) launch_walls_t<2, 0>(t, tl, wall_tiles, d_nwall, tiles_upper, st);
    else launch_walls_t<2, 1>(t, tl, wall_tiles, d_nwall, tiles_upper, st);
  } else {
    if (kern == 0) launch_walls_t<3, 0>(t, tl, wall_tiles, d_nwall, tiles_upper, st);
    else launch_walls_t<3, 1>(t, tl, wall_tiles, d_nwall, tiles_upper, st);
  }
  CKL();
  prof_end();
  ++launches;
}

// <grad rho>^L of every particle into gradrho (after the wall pass has set the walls' density)
void Scene::grad_pass(const TravArgs& t, const Tile* tl, const int* ntl) {
  if (!gradrho) gradrho = (float4*)mem.get(sizeof(float4) * N);
  prof_begin(5);
  if (D == 2) {
    if (kern == 0) launch_grad_t<2, 0>(t, tl, ntl, tiles_upper, gradrho, st);
    else launch_grad_t<2, 1>(t, tl, ntl, tiles_upper, gradrho, st);
  } else {
    if (kern == 0) launch_grad_t<3, 0>(t, tl, ntl, tiles_upper, gradrho, st);
    else launch_grad_t<3, 1>(t, tl, ntl, tiles_upper, gradrho, st);
  }
  CKL();
  prof_end();
  ++launches;
}

void Scene::passes_before_sweep(const TravArgs& t_in, const Tile* tl, const int* ntl, bool fused_walls) {
  if (!tl) {
    tl = tiles;
    ntl = d_ntiles;
  }
  TravArgs t = t_in;
  t.pair_count = nullptr;  // pair counts are those of the sweep (fluid targets) only
  // the step's order (Sec. 3.4): summation density of the fluid, then the walls' pressure from
  // the fluid's, then the gradients that need both
  if (summation) {
    prof_begin(3);
    if (D == 2) {
      if (kern == 0) launch_density_t<2, 0>(t, tl, ntl, tiles_upper, st);
      else launch_density_t<2, 1>(t, tl, ntl, tiles_upper, st);
    } else {
      if (kern == 0) launch_density_t<3, 0>(t, tl, ntl, tiles_upper, st);
      else launch_density_t<3, 1>(t, tl, ntl, tiles_upper, st);
    }
    CKL();
    prof_end();
    ++launches;
  }
  if (any_walls && !fused_walls) walls_pass(t, tl);
  if (renorm) grad_pass(t, tl, ntl);
}

void Scene::sweep(const TravArgs& t, const Arrays& out, const Tile* tl, const int* ntl, bool fused_walls,
                  const Displace* disp) {
  if (!tl) {
    tl = tiles;
    ntl = d_ntiles;
  }
  prof_begin(0);
  const Displace dp = disp ? *disp
                    : dev_policy ? Displace{xbuild, &d_ctl->maxr, inv_r2, use_coop ? d_ctl : nullptr, interval}
                                 : Displace{nullptr, nullptr, 0.f, nullptr, 0};
  const float4* g = renorm ? gradrho : nullptr;
  if (fused_walls) {
    if (D == 2) {
      if (kern == 0) launch_walls_sweep_t<2, 0>(t, wall_plans, fluid_plans, d_nwall, tiles_upper, out, dp, st);
      else launch_walls_sweep_t<2, 1>(t, wall_plans, fluid_plans, d_nwall, tiles_upper, out, dp, st);
    } else {
      if (kern == 0) launch_walls_sweep_t<3, 0>(t, wall_plans, fluid_plans, d_nwall, tiles_upper, out, dp, st);
      else launch_walls_sweep_t<3, 1>(t, wall_plans, fluid_plans, d_nwall, tiles_upper, out, dp, st);
    }
  } else if (D == 2) {
    if (kern == 0) launch_sweep_t<2, 0>(t, tl, ntl, tiles_upper, out, dp, g, st);
    else launch_sweep_t<2, 1>(t, tl, ntl, tiles_upper, out, dp, g, st);
  } else {
    if (kern == 0) launch_sweep_t<3, 0>(t, tl, ntl, tiles_upper, out, dp, g, st);
    else launch_sweep_t<3, 1>(t, tl, ntl, tiles_upper, out, dp, g, st);
  }
  CKL();
  prof_end();
  launches += fused_walls ? 1 : sweep_kernels(D, N, t.packed);
}

// Particle shifting at the end of the step: from buf[cur] (the sweep's result, on cells valid
// for it) into the other buffer.
void Scene::shift_pass() {
  prof_begin(6);
  TravArgs t = trav(buf[cur], keys_sorted, cell_off);
  t.pair_count = nullptr;  // pair counts are those of the sweep
  const Displace dp = dev_policy ? Displace{xbuild, &d_ctl->maxr, inv_r2, use_coop ? d_ctl : nullptr, interval}
                                 : Displace{nullptr, nullptr, 0.f, nullptr, 0};
  if (D == 2) {
    if (kern == 0) launch_shift_t<2, 0>(t, tiles, d_ntiles, tiles_upper, buf[1 - cur], dp, st);
    else launch_shift_t<2, 1>(t, tiles, d_ntiles, tiles_upper, buf[1 - cur], dp, st);
  } else {
    if (kern == 0) launch_shift_t<3, 0>(t, tiles, d_ntiles, tiles_upper, buf[1 - cur], dp, st);
    else launch_shift_t<3, 1>(t, tiles, d_ntiles, tiles_upper, buf[1 - cur], dp, st);
  }
  CKL();
  prof_end();
  ++launches;
  cur = 1 - cur;
}

// Rebuild launched by the host (eager steps, cells needed by a query): permute into the other
// buffer; the device-side policy counters restart from this rebuild.
void Scene::host_rebuild() {
  auto kp = rebuild(buf[cur], buf[1 - cur], nullptr, nullptr, cell_off, nullptr, nullptr, xorder ? bin_off : nullptr);
  keys_sorted = kp.first;
  perm = kp.second;
  cur = 1 - cur;
  cells_valid = true;
  steps_since_build = 0;
  if (!capturing) ++host_rebuilds;  // captured rebuilds are counted per graph launch
  if (dev_policy) {  // since = 0, maxr = 0, no rebuild pending
    CK(cudaMemsetAsync(d_ctl, 0, 2 * sizeof(int), st));
    CK(cudaMemsetAsync(&d_ctl->flag, 0, sizeof(int), st));
  }
}

// One forward step on the scene's own buffers.  Eager steps rebuild every time (the host does
// not see the displacements) unless eager_dev is set, where the device decides as in captured
// steps (the cooperative rebuild launch needs no host decision); captured steps of a scene with
// a Verlet skin decide on the device.
void Scene::step_once() {
  if (dev_policy && cells_valid && (capturing || (eager_dev && use_coop))) {
    if (use_coop)
      step_coop();
    else
      step_conditional();
    return;
  }
  host_rebuild();
  TravArgs t = trav(buf[cur], keys_sorted, cell_off, xorder ? bin_off : nullptr);
  passes_before_sweep(t, nullptr, nullptr, walls_in_sweep());
  sweep(t, buf[1 - cur], nullptr, nullptr, walls_in_sweep());
  cur = 1 - cur;
  ++steps_since_build;
  if (shifting) {  // the shift needs the neighbours of the swept positions
    host_rebuild();
    shift_pass();
  }
}

// A captured step whose rebuild is a conditional graph node: a one-thread kernel decides
// (interval reached, or the previous sweep saw a displacement beyond skin/2), the node's body
// sorts and permutes into the other buffer and copies the result back, so the buffer parity of
// the step does not depend on the decision.
void Scene::step_conditional() {
  cond_rebuild(1);
  TravArgs t = trav(buf[cur], keys_sorted, cell_off, xorder ? bin_off : nullptr);
  passes_before_sweep(t, nullptr, nullptr, walls_in_sweep());
  sweep(t, buf[1 - cur], nullptr, nullptr, walls_in_sweep());
  cur = 1 - cur;
  if (shifting) {
    cond_rebuild(0);
    shift_pass();
  }
}

// The conditional rebuild node (count: whether a sweep follows and uses the cells).
void Scene::cond_rebuild(int count) {
  prof_begin(1);
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* ed = nullptr;
  size_t nd = 0;
  CK(cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, &ed, &nd));
  cudaGraphConditionalHandle h;
  CK(cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault));
  launch_rebuild_decide(d_ctl, interval, count, h, st);
  CKL();
  ++launches;
  CK(cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, &ed, &nd));
  cudaGraphNodeParams np{};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeIf;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  CK(cudaGraphAddNode(&node, g, deps, ed, nd, &np));
  cudaGraph_t body = np.conditional.phGraph_out[0];
  if (!st_body) CK(cudaStreamCreateWithFlags(&st_body, cudaStreamNonBlocking));
  CK(cudaStreamBeginCaptureToGraph(st_body, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  const long long l0 = launches;
  std::swap(st, st_body);
  in_body = true;
  try {
    rebuild(buf[cur], buf[1 - cur], nullptr, nullptr, cell_off, nullptr, nullptr, xorder ? bin_off : nullptr);
    if (D == 2)
      launch_copy_state<2>(N, buf[1 - cur], buf[cur], st);
    else
      launch_copy_state<3>(N, buf[1 - cur], buf[cur], st);
    CKL();
    ++launches;
  } catch (...) {
    in_body = false;
    std::swap(st, st_body);
    cudaGraph_t dummy;
    cudaStreamEndCapture(st_body, &dummy);
    throw;
  }
  in_body = false;
  std::swap(st, st_body);
  body_launches = launches - l0;
  launches = l0;
  cudaGraph_t dummy;
  CK(cudaStreamEndCapture(st_body, &dummy));
  CK(cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  prof_end();
  keys_sorted = (passes % 2 == 0) ? kA : kB;
  perm = (passes % 2 == 0) ? vA : vB;
}

// A captured step whose rebuild is one cooperative launch that returns at once unless the
// previous sweep asked for a rebuild; when it rebuilds it sorts and permutes into the other
// buffer and copies the result back, so the buffer parity does not depend on the decision.
RebuildArgs Scene::coop_args(const Arrays& in, const Arrays& out, int* off, const int* flag, int copy_back) {
  RebuildArgs r{};
  r.segs = dseg;
  r.S = S;
  r.N = N;
  r.C = C_tot;
  r.passes = passes;
  r.nb = (N + 2047) / 2048;
  r.in = in;
  r.out = out;
  r.copy_back = copy_back;
  r.kA = kA; r.vA = vA; r.kB = kB; r.vB = vB;
  r.hist = scratch;
  r.sums = scratch + (sort_scratch_words(N) - 2048 - 64);
  r.off = off;
  r.boff = xorder ? bin_off : nullptr;
  r.xb = xbuild;
  r.line_base = line_base;
  r.n_lines = n_lines;
  r.tiles = tiles;
  r.ntiles = d_ntiles;
  r.wall_list = any_walls ? wall_tiles : nullptr;
  r.wall_plans = any_walls ? wall_plans : nullptr;
  r.fluid_plans = any_walls ? fluid_plans : nullptr;
  r.nwall = any_walls ? d_nwall : nullptr;
  r.flag = flag;
  r.ctl = flag ? d_ctl : nullptr;
  r.bar = d_bar;
  r.status = d_status;
  return r;
}

void Scene::step_coop() {
  coop_rebuild();
  TravArgs t = trav(buf[cur], keys_sorted, cell_off, xorder ? bin_off : nullptr);
  passes_before_sweep(t, nullptr, nullptr, walls_in_sweep());
  sweep(t, buf[1 - cur], nullptr, nullptr, walls_in_sweep());
  cur = 1 - cur;
  if (shifting) {  // the sweep's last CTA has decided whether the shift needs new cells
    coop_rebuild();
    shift_pass();
  }
}

void Scene::coop_rebuild() {
  prof_begin(1);
  const RebuildArgs r = coop_args(buf[cur], buf[1 - cur], cell_off, &d_ctl->flag, 1);
  CK(D == 2 ? launch_rebuild_coop<2>(r, coop_grid, st) : launch_rebuild_coop<3>(r, coop_grid, st));
  ++launches;
  prof_end();
  keys_sorted = (passes % 2 == 0) ? kA : kB;
  perm = (passes % 2 == 0) ? vA : vB;
}

// Host-side replay of the buffer schedule of one captured step (graph bookkeeping).
void Scene::advance_schedule() {
  if (!dev_policy) cur = 1 - cur;  // the rebuild's permute
  cur = 1 - cur;                   // the sweep
  if (shifting) {
    if (!dev_policy) cur = 1 - cur;  // the rebuild before the shift
    cur = 1 - cur;                   // the shift
  }
  cells_valid = true;
  keys_sorted = (passes % 2 == 0) ? kA : kB;
  perm = (passes % 2 == 0) ? vA : vB;
}

void Scene::steps(int n) {
  need_ghosts();
  if (n <= 0) return;
  CK(cudaMemsetAsync(d_pairs, 0, sizeof(unsigned long long), st));
  launches = 0;
  const int chunk = std::min(graph_chunk, n);
  steps_total += n;
  if (dev_policy) CK(cudaMemsetAsync(&d_ctl->call_rebuilds, 0, sizeof(long long), st));
  if (!use_graphs) {
    for (int k = 0; k < n; ++k) step_once();
    last_steps = n;
    launches_total += launches;
    return;
  }
  int done = 0;
  long long per_chunk = 0;
  if (dev_policy && !cells_valid) host_rebuild();
  while (done < n) {
    const int c = std::min(chunk, n - done);  // the last graph takes the remainder
    GraphKey key{c, cur, dev_policy ? 1 : 0, profiling ? 1 : 0};
    auto it = graphs.find(key);
    // capture records the launches of `chunk` steps without running them; the host-side
    // schedule (buffer parity, rebuild counter, sorted-key pointers) advances exactly as in
    // an eager run, so it is simply kept after the capture.
    long long l0 = launches;
    if (it == graphs.end()) {
      cudaGraph_t g;
      capturing = true;
      CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
      try {
        for (int k = 0; k < c; ++k) step_once();
      } catch (...) {
        cudaStreamEndCapture(st, &g);
        capturing = false;
        throw;
      }
      CK(cudaStreamEndCapture(st, &g));
      capturing = false;
      // locate the event-record nodes of the timed launches
      std::vector<GraphProfNode> pn;
      if (!capture_events.empty()) {
        size_t nn = 0;
        CK(cudaGraphGetNodes(g, nullptr, &nn));
        std::vector<cudaGraphNode_t> nodes(nn);
        CK(cudaGraphGetNodes(g, nodes.data(), &nn));
        for (auto& ce : capture_events) {
          GraphProfNode gn{ce.cls, nullptr, nullptr};
          for (auto nd : nodes) {
            cudaGraphNodeType t;
            CK(cudaGraphNodeGetType(nd, &t));
            if (t != cudaGraphNodeTypeEventRecord) continue;
            cudaEvent_t ev;
            CK(cudaGraphEventRecordNodeGetEvent(nd, &ev));
            if (ev == ce.a) gn.a = nd;
            if (ev == ce.b) gn.b = nd;
          }
          if (gn.a && gn.b) pn.push_back(gn);
          event_pool.push_back(ce.a);
          event_pool.push_back(ce.b);
        }
        capture_events.clear();
      }
      cudaGraphExec_t ge;
      CK(cudaGraphInstantiate(&ge, g, 0));
      if (pn.empty())
        cudaGraphDestroy(g);
      else
        graph_templates.push_back(g);
      graphs[key] = ge;
      graph_prof[key] = pn;
      it = graphs.find(key);
      per_chunk = launches - l0;
      graph_launch_count[key] = per_chunk;
    } else {
      for (int k = 0; k < c; ++k) advance_schedule();
      launches += graph_launch_count[key];
    }
    if (!dev_policy) host_rebuilds += c;  // every captured step rebuilds
    for (auto& gn : graph_prof[key]) {
      ProfEvent e;
      e.cls = gn.cls;
      e.a = take_event();
      e.b = take_event();
      CK(cudaGraphExecEventRecordNodeSetEvent(it->second, gn.a, e.a));
      CK(cudaGraphExecEventRecordNodeSetEvent(it->second, gn.b, e.b));
      prof_events.push_back(e);
    }
    CK(cudaGraphLaunch(it->second, st));
    done += c;
  }
  last_steps = n;
  launches_total += launches;
}

void Scene::ensure_cells() {
  if (cells_valid) return;
  host_rebuild();
}

// ---------------------------------------------------------------- adjoint tape
void Scene::rollout(int n, int k) {
  need_ghosts();
  if (n < 1 || k < 1) einval("n_steps and ckpt_every must be >= 1");
  if (renorm) einval("the renormalised diffusion (SPH_DIFFUSION_RENORM) has no adjoint; use sph_step");
  if (shifting) einval("particle shifting has no adjoint; use sph_step");
  tape_n = n;
  tape_k = k;
  int ncp = (n + k - 1) / k;
  if ((int)ckpts.size() < ncp) {
    while ((int)ckpts.size() < ncp) {
      Arrays a;
      alloc_arrays(a);
      ckpts.push_back(a);
    }
  }
  // segment by segment: checkpoint, then the segment's steps exactly as sph_step runs them
  // (graph chunks, the same rebuild schedule), starting from a fresh build like the replay
  long long seg_launches = 0;
  int64_t r0 = 0, r1 = 0;
  if (dev_policy) stats(nullptr, &r0, nullptr);
  for (int s0 = 0; s0 < n; s0 += k) {
    copy_arrays(ckpts[s0 / k], buf[cur]);
    cells_valid = false;
    steps(std::min(k, n - s0));
    seg_launches += launches;
  }
  launches = seg_launches;  // (pair counts: those of the last segment's steps)
  tape_valid = true;
  if (dev_policy) {
    // the adjoint's replay starts from three quarters of the rollout's mean rebuild interval
    // (or the caller's choice)
    stats(nullptr, &r1, nullptr);
    const int64_t rb = std::max<int64_t>(1, r1 - r0);
    replay_k = replay_k_user > 0 ? replay_k_user
                                 : (int)std::max<int64_t>(1, std::min<int64_t>(16, (3 * (int64_t)n) / (4 * rb)));
  }
}

void Scene::alloc_tape(int k) {
  if (tape_cap >= k) return;
  for (int b = 0; b < 2; ++b) {
    while ((int)tapes[b].size() < k + 1) {
      TapeSlot t;
      alloc_arrays(t.a);
      t.keys = (uint32_t*)mem.get(4 * (size_t)N);
      t.perm = (uint32_t*)mem.get(4 * (size_t)N);
      t.off = (int*)mem.get(sizeof(int) * ((size_t)C_tot + 1));
      t.tiles = (Tile*)mem.get(sizeof(Tile) * (size_t)tiles_upper);
      t.ntiles = (int*)mem.get(sizeof(int) * 2);
      t.boff = xorder ? (int*)mem.get(sizeof(int) * ((size_t)C_tot * kXBins + 1)) : nullptr;
      tapes[b].push_back(t);
    }
  }
  if (!adj_alloc) {
    for (int q = 0; q < 2; ++q) {
      XB[q] = (float4*)mem.get(sizeof(float4) * N);
      VB[q] = (float4*)mem.get(sizeof(float4) * N);
    }
    Sd = (float4*)mem.get(sizeof(float4) * N);
    Pp = (float*)mem.get(sizeof(float) * N);
    adj_rows = (float*)mem.get(sizeof(float) * (2 * (size_t)N * D + (size_t)N + 64));
    d_replay_flag = (int*)mem.get(sizeof(int) * 4);
    d_replay_maxr = (unsigned*)mem.get(sizeof(unsigned) * 2);
    CK(cudaMemsetAsync(d_replay_flag, 0, sizeof(int) * 4, st));
    CK(cudaMemsetAsync(d_replay_maxr, 0, sizeof(unsigned) * 2, st));
    nu_acc = (double*)mem.get(sizeof(double) * (size_t)N);
    alloc_arrays(scratch_arr);
    rep_out[0] = scratch_arr;
    alloc_arrays(rep_out[1]);
    alloc_arrays(ckpt_work);
    d_tile_ctr_b = (int*)mem.get(sizeof(int) * 4);
    CK(cudaMemsetAsync(d_tile_ctr_b, 0, sizeof(int) * 4, st));  // tiled kernels leave it zeroed
    adj_alloc = true;
  }
  tape_cap = k;
}

// Replay one segment of L steps forward from ckpt_work, keeping each step's sweep input in the
// tape.  The cells are rebuilt at the segment's first step and every K steps (K = 1: every step);
// a slot between rebuilds shares the cells of the last rebuild, and the sweep before it writes the
// slot directly.  With K > 1 the sweeps measure the displacement since the last rebuild, and a
// step whose successor does not rebuild sets d_replay_flag when it exceeds the skin's half: the
// caller then replays the segment with K = 1.
void Scene::adjoint_replay(int L, int K, int b) {
  std::vector<TapeSlot>& tape = tapes[b];
  const Arrays* prev = &ckpt_work;
  int r = 0;
  for (int s = 0; s < L; ++s) {
    TapeSlot& slot = tape[s];
    if (s % K == 0) {
      rebuild(*prev, slot.a, slot.keys, slot.perm, slot.off, slot.tiles, slot.ntiles, slot.boff);  // kept in the slot
      r = s;
    }
    const TapeSlot& cells = tape[r];
    TravArgs t = trav(slot.a, cells.keys, cells.off, cells.boff);
    passes_before_sweep(t, cells.tiles, cells.ntiles);
    const bool next_rebuilds = s + 1 == L || (s + 1) % K == 0;
    const Arrays& out = next_rebuilds ? rep_out[b] : tape[s + 1].a;
    if (K > 1) {
      const Displace dp{xbuild, d_replay_maxr, inv_r2, nullptr, interval, next_rebuilds ? d_replay_flag + 1 : d_replay_flag};
      sweep(t, out, cells.tiles, cells.ntiles, false, &dp);
    } else {
      sweep(t, out, cells.tiles, cells.ntiles);
    }
    prev = &rep_out[b];
  }
}

// The adjoint steps of a replayed segment backwards (rebuild every K steps, as replayed).  The
// adjoint state enters and leaves in XB[0]/VB[0].
void Scene::adjoint_backward(int L, int K, int b) {
  std::vector<TapeSlot>& tape = tapes[b];
  int q = 0;
  for (int s = L - 1; s >= 0; --s) {
    TapeSlot& slot = tape[s];
    const TapeSlot& cells = tape[(s / K) * K];
    if (D == 2)
      launch_adj_seed<2>(dseg, N, slot.a, XB[q], VB[q], Sd, Pp, st);
    else
      launch_adj_seed<3>(dseg, N, slot.a, XB[q], VB[q], Sd, Pp, st);
    CKL();
    TravArgs t = trav(slot.a, cells.keys, cells.off);
    t.pair_count = nullptr;
    t.tile_ctr = d_tile_ctr_b;  // the next segment's replay may be running on st_rep
    prof_begin(4);
    if (D == 2) {
      if (kern == 0)
        launch_adj_t<2, 0>(t, cells.tiles, cells.ntiles, tiles_upper, Sd, Pp, XB[q], VB[q], XB[1 - q], VB[1 - q], nu_acc, st);
      else
        launch_adj_t<2, 1>(t, cells.tiles, cells.ntiles, tiles_upper, Sd, Pp, XB[q], VB[q], XB[1 - q], VB[1 - q], nu_acc, st);
    } else {
      if (kern == 0)
        launch_adj_t<3, 0>(t, cells.tiles, cells.ntiles, tiles_upper, Sd, Pp, XB[q], VB[q], XB[1 - q], VB[1 - q], nu_acc, st);
      else
        launch_adj_t<3, 1>(t, cells.tiles, cells.ntiles, tiles_upper, Sd, Pp, XB[q], VB[q], XB[1 - q], VB[1 - q], nu_acc, st);
    }
    CKL();
    prof_end();
    q = 1 - q;
    launches += 2;  // seed, adjoint sweep
    if (summation) {  // the density adjoint left in XB.w passes to the positions
      if (D == 2) {
        if (kern == 0) launch_adj_dens_t<2, 0>(t, cells.tiles, cells.ntiles, tiles_upper, XB[q], VB[q], XB[1 - q], VB[1 - q], st);
        else launch_adj_dens_t<2, 1>(t, cells.tiles, cells.ntiles, tiles_upper, XB[q], VB[q], XB[1 - q], VB[1 - q], st);
      } else {
        if (kern == 0) launch_adj_dens_t<3, 0>(t, cells.tiles, cells.ntiles, tiles_upper, XB[q], VB[q], XB[1 - q], VB[1 - q], st);
        else launch_adj_dens_t<3, 1>(t, cells.tiles, cells.ntiles, tiles_upper, XB[q], VB[q], XB[1 - q], VB[1 - q], st);
      }
      CKL();
      q = 1 - q;
      ++launches;
    }
    if (s % K == 0) {  // the step's rebuild permuted the state: back to the previous order
      launch_adj_unpermute(N, slot.perm, XB[q], VB[q], XB[1 - q], VB[1 - q], st);
      CKL();
      q = 1 - q;
      ++launches;
    }
  }
  if (q != 0) {  // back into XB[0]/VB[0]
    CK(cudaMemcpyAsync(XB[0], XB[1], sizeof(float4) * N, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(VB[0], VB[1], sizeof(float4) * N, cudaMemcpyDeviceToDevice, st));
  }
}

// Runs (or captures and replays) one part of a segment: part 0 the forward replay, 1 the adjoint.
void Scene::adjoint_part(int part, int L, int K, int b) {
  if (!use_graphs || profiling) {
    if (part == 0) adjoint_replay(L, K, b);
    else adjoint_backward(L, K, b);
    return;
  }
  const long long key = ((long long)part << 41) | ((long long)b << 40) | ((long long)K << 20) | (long long)L;
  auto it = adj_graphs.find(key);
  if (it == adj_graphs.end()) {
    const long long l0 = launches;
    cudaGraph_t g;
    capturing = true;
    CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    try {
      if (part == 0) adjoint_replay(L, K, b);
      else adjoint_backward(L, K, b);
    } catch (...) {
      cudaStreamEndCapture(st, &g);
      capturing = false;
      throw;
    }
    CK(cudaStreamEndCapture(st, &g));
    capturing = false;
    cudaGraphExec_t ge;
    CK(cudaGraphInstantiate(&ge, g, 0));
    cudaGraphDestroy(g);
    it = adj_graphs.emplace(key, std::make_pair(ge, launches - l0)).first;
  } else {
    launches += it->second.second;
  }
  CK(cudaGraphLaunch(it->second.first, st));
}

// The forward replay of segment sgi into tape b, on the scene's current stream: from a working
// copy of the segment's checkpoint (so that one captured graph per segment length serves every
// segment), rebuilding every replay_k steps when the skin allows; a segment whose displacements
// outgrew the skin is replayed again with a rebuild every step (and later segments try half the
// interval).  Returns the rebuild interval the tape was recorded with.
int Scene::adjoint_replay_segment(int sgi, int b) {
  const int t0 = sgi * tape_k, t1 = std::min(tape_n, t0 + tape_k);
  const int L = t1 - t0;
  if (D == 2)
    launch_copy_state<2>(N, ckpts[sgi], ckpt_work, st);
  else
    launch_copy_state<3>(N, ckpts[sgi], ckpt_work, st);
  CKL();
  ++launches;
  int K = std::max(1, std::min(replay_k, L));
  if (K > 1) CK(cudaMemsetAsync(d_replay_flag, 0, sizeof(int) * 2, st));
  adjoint_part(0, L, K, b);
  if (K > 1) {
    int flag = 0;
    CK(cudaMemcpyAsync(&flag, d_replay_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (flag) {
      ++replay_fallbacks;
      replay_k = std::max(1, replay_k / 2);
      K = 1;
      adjoint_part(0, L, K, b);
    }
  }
  return K;
}

void Scene::adjoint(const float* xb, const float* vb, const float* rb, float* xb0, float* vb0, float* rb0, double* nub,
                    int is_dev) {
  if (!tape_valid) einval("sph_adjoint needs a preceding sph_rollout on this scene");
  if (any_walls) einval("the adjoint supports scenes without wall particles");
  const int n = tape_n, k = tape_k;
  alloc_tape(k);
  launches = 0;
  // seeds of the final state, scattered into the final storage order
  const size_t nd = (size_t)nf_total * D;
  const float *dxb = xb, *dvb = vb, *drb = rb;
  if (!is_dev) {
    float* p = (float*)mem_tmp(sizeof(float) * (2 * nd + nf_total + 64));
    if (xb) { CK(cudaMemcpyAsync(p, xb, 4 * nd, cudaMemcpyHostToDevice, st)); dxb = p; }
    if (vb) { CK(cudaMemcpyAsync(p + nd, vb, 4 * nd, cudaMemcpyHostToDevice, st)); dvb = p + nd; }
    if (rb) { CK(cudaMemcpyAsync(p + 2 * nd, rb, 4 * (size_t)nf_total, cudaMemcpyHostToDevice, st)); drb = p + 2 * nd; }
  }
  int q = 0;
  // the adjoint state is carried in storage order; each segment's replay may store the particles
  // in another order than the forward rollout did (its rebuild schedule differs), so the state
  // enters each segment through the original order: the seeds after the last segment's replay,
  // the running adjoint by a store / load through the rows at every later segment
  float* rows = adj_rows;
  // dL/dnu: each adjoint sweep adds its particles' terms into their storage slots (nu_acc), and
  // one deterministic per-scene sum over the slots after the last segment gives the total (the
  // slots' order changes at rebuilds, which only regroups the same terms)
  CK(cudaMemsetAsync(d_nubar, 0, sizeof(double) * S, st));
  CK(cudaMemsetAsync(nu_acc, 0, sizeof(double) * (size_t)N, st));
  const int ncp = (n + k - 1) / k;
  // The segments' replays run on st_rep, one segment ahead of the reverse pass on st: while the
  // reverse pass of segment sgi reads tape sgi % 2, the replay of segment sgi - 1 fills the other
  // tape (each pass alone leaves most of the GPU idle at the sizes the adjoint is used at).  A
  // replay waits for the reverse pass that last read its tape; a reverse pass waits for its replay.
  if (!st_rep) {  // with the priority of the scene's stream
    int prio = 0;
    CK(cudaStreamGetPriority(st, &prio));
    CK(cudaStreamCreateWithPriority(&st_rep, cudaStreamNonBlocking, prio));
  }
  for (int b = 0; b < 2; ++b) {
    if (!ev_rep[b]) CK(cudaEventCreateWithFlags(&ev_rep[b], cudaEventDisableTiming));
    if (!ev_free[b]) CK(cudaEventCreateWithFlags(&ev_free[b], cudaEventDisableTiming));
    CK(cudaEventRecord(ev_free[b], st));  // the replays start after the work queued on st so far
  }
  auto replay_beside = [&](int sgi) {
    const int b = sgi & 1;
    CK(cudaStreamWaitEvent(st_rep, ev_free[b], 0));
    std::swap(st, st_rep);
    int K = 1;
    try {
      K = adjoint_replay_segment(sgi, b);
    } catch (...) {
      std::swap(st, st_rep);
      throw;
    }
    std::swap(st, st_rep);
    CK(cudaEventRecord(ev_rep[b], st_rep));
    return K;
  };
  int K = replay_beside(ncp - 1);
  for (int sgi = ncp - 1; sgi >= 0; --sgi) {
    const int b = sgi & 1;
    const int L = std::min(n, sgi * k + k) - sgi * k;
    CK(cudaStreamWaitEvent(st, ev_rep[b], 0));
    // the adjoint of the segment's final state, in the order of the replay's last sweep output
    const float *lx = dxb, *lv = dvb, *lr = drb;
    if (sgi != ncp - 1) {  // the running adjoint, in the order of the checkpoint after this segment
      if (D == 2)
        launch_adj_store<2>(N, ckpts[sgi + 1].meta, d_orig_base, XB[0], VB[0], rows, rows + nd, rows + 2 * nd, st);
      else
        launch_adj_store<3>(N, ckpts[sgi + 1].meta, d_orig_base, XB[0], VB[0], rows, rows + nd, rows + 2 * nd, st);
      CKL();
      lx = rows;
      lv = rows + nd;
      lr = rows + 2 * nd;
      ++launches;
    }
    if (D == 2)
      launch_adj_load<2>(N, rep_out[b].meta, d_orig_base, lx, lv, lr, XB[0], VB[0], st);
    else
      launch_adj_load<3>(N, rep_out[b].meta, d_orig_base, lx, lv, lr, XB[0], VB[0], st);
    CKL();
    ++launches;
    adjoint_part(1, L, K, b);
    CK(cudaEventRecord(ev_free[b], st));
    if (sgi > 0) K = replay_beside(sgi - 1);
  }
  // XB[q] is in the storage order of checkpoint 0; deliver in original order
  float* oxb = xb0;
  float* ovb = vb0;
  float* orb = rb0;
  float* stage = nullptr;
  if (!is_dev) {
    stage = (float*)mem_tmp(sizeof(float) * (2 * nd + nf_total + 64));
    oxb = xb0 ? stage : nullptr;
    ovb = vb0 ? stage + nd : nullptr;
    orb = rb0 ? stage + 2 * nd : nullptr;
  }
  if (D == 2)
    launch_adj_store<2>(N, ckpts[0].meta, d_orig_base, XB[q], VB[q], oxb, ovb, orb, st);
  else
    launch_adj_store<3>(N, ckpts[0].meta, d_orig_base, XB[q], VB[q], oxb, ovb, orb, st);
  CKL();
  launch_sum_segments(nu_acc, dseg, S, sum_nch, sum_chunk, sum_ctr, d_nubar, st);
  CKL();
  launches += 2;
  // the replay reused the sort buffers: the live state must rebuild before its next step
  cells_valid = false;
  launches_total += launches;
  if (!is_dev) {
    if (xb0) CK(cudaMemcpyAsync(xb0, oxb, 4 * nd, cudaMemcpyDeviceToHost, st));
    if (vb0) CK(cudaMemcpyAsync(vb0, ovb, 4 * nd, cudaMemcpyDeviceToHost, st));
    if (rb0) CK(cudaMemcpyAsync(rb0, orb, 4 * (size_t)nf_total, cudaMemcpyDeviceToHost, st));
  }
  if (nub) CK(cudaMemcpyAsync(nub, d_nubar, sizeof(double) * S, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
}

// ---------------------------------------------------------------- outputs
void Scene::get_state(float* x, float* v, float* rho, int is_dev) {
  const size_t nd = (size_t)N * D;
  float *ox = x, *ov = v, *orh = rho;
  if (!is_dev) {
    float* p = (float*)mem_tmp(sizeof(float) * (2 * nd + N + 64));
    ox = x ? p : nullptr;
    ov = v ? p + nd : nullptr;
    orh = rho ? p + 2 * nd : nullptr;
  }
  if (D == 2)
    launch_download<2>(N, buf[cur], d_orig_base, ox, ov, orh, st);
  else
    launch_download<3>(N, buf[cur], d_orig_base, ox, ov, orh, st);
  CKL();
  if (!is_dev) {
    if (x) CK(cudaMemcpyAsync(x, ox, 4 * nd, cudaMemcpyDeviceToHost, st));
    if (v) CK(cudaMemcpyAsync(v, ov, 4 * nd, cudaMemcpyDeviceToHost, st));
    if (rho) CK(cudaMemcpyAsync(rho, orh, 4 * (size_t)N, cudaMemcpyDeviceToHost, st));
  }
  check_status();
}

// The status words (synchronises): [0] error bits, then one word per scene of the batch (bit 0: that
// scene became unstable).
std::vector<int> Scene::status_words() {
  std::vector<int> h(4 + (size_t)S);
  CK(cudaMemcpyAsync(h.data(), d_status, sizeof(int) * h.size(), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return h;
}

// Clear the instability marks (the caller has taken the unstable scenes out).
void Scene::clear_unstable() {
  CK(cudaMemsetAsync(d_status, 0, sizeof(int), st));
  CK(cudaMemsetAsync(d_status + 4, 0, sizeof(int) * (size_t)S, st));
}

void Scene::check_status() {
  int h = 0;
  CK(cudaMemcpyAsync(&h, d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (h & 2) {
    set_err("a bounded device wait gave up (a grid barrier of the cooperative rebuild, a sweep tile waiting for the wall tasks, or a warp waiting for its CTA's tile chunk)");
    throw Fail{SPH_EINTERNAL};
  }
  if (h & 1) {
    set_err("unstable state: non-finite values or density outside [0.5, 2] rho0");
    throw Fail{SPH_EUNSTABLE};
  }
}

void Scene::rates(float* a, float* drho, float* rho, int is_dev) {
  need_ghosts();
  // summation density / walls modify the records in place: work on a copy
  ensure_cells();
  if (!adj_alloc) alloc_tape(1);
  copy_arrays(scratch_arr, buf[cur]);
  TravArgs t = trav(scratch_arr, keys_sorted, cell_off);
  passes_before_sweep(t);
  const size_t nd = (size_t)nf_total * D;
  float* p = (float*)mem_tmp(sizeof(float) * (nd + 2 * (size_t)nf_total + 64));
  RateOut ro;
  ro.a = p;
  ro.drho = p + nd;
  ro.rho = p + nd + nf_total;
  // outputs are indexed by fluid rows: original index + scene base among fluid rows
  std::vector<int> fbase(S);
  int acc = 0;
  for (int s = 0; s < S; ++s) {
    fbase[s] = acc;
    acc += segs[s].nf;
  }
  if (!d_fluid_base) d_fluid_base = (int*)mem.get(sizeof(int) * S);
  CK(cudaMemcpyAsync(d_fluid_base, fbase.data(), sizeof(int) * S, cudaMemcpyHostToDevice, st));
  ro.orig_base = d_fluid_base;
  const float4* g = renorm ? gradrho : nullptr;
  if (D == 2) {
    if (kern == 0) launch_rates_t<2, 0>(t, tiles, d_ntiles, tiles_upper, ro, g, st);
    else launch_rates_t<2, 1>(t, tiles, d_ntiles, tiles_upper, ro, g, st);
  } else {
    if (kern == 0) launch_rates_t<3, 0>(t, tiles, d_ntiles, tiles_upper, ro, g, st);
    else launch_rates_t<3, 1>(t, tiles, d_ntiles, tiles_upper, ro, g, st);
  }
  CKL();
  cudaMemcpyKind kind = is_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (a) CK(cudaMemcpyAsync(a, ro.a, 4 * nd, kind, st));
  if (drho) CK(cudaMemcpyAsync(drho, ro.drho, 4 * (size_t)nf_total, kind, st));
  if (rho) CK(cudaMemcpyAsync(rho, ro.rho, 4 * (size_t)nf_total, kind, st));
  CK(cudaStreamSynchronize(st));
}

// <grad rho>^L at the current state in original order (all particles), on a copy of the records
// (the wall pass writes the walls' density in place).
void Scene::density_gradient(float* grad, int is_dev) {
  need_ghosts();
  ensure_cells();
  if (!adj_alloc) alloc_tape(1);
  copy_arrays(scratch_arr, buf[cur]);
  TravArgs t = trav(scratch_arr, keys_sorted, cell_off);
  t.pair_count = nullptr;
  if (any_walls) walls_pass(t, tiles);
  grad_pass(t, tiles, d_ntiles);
  const size_t nd = (size_t)N * D;
  float* out = is_dev ? grad : (float*)mem_tmp(sizeof(float) * (nd + 64));
  // the adjoint's unpermuting store writes the xyz of a float4 array to original rows
  if (D == 2)
    launch_adj_store<2>(N, scratch_arr.meta, d_orig_base, gradrho, gradrho, out, nullptr, nullptr, st);
  else
    launch_adj_store<3>(N, scratch_arr.meta, d_orig_base, gradrho, gradrho, out, nullptr, nullptr, st);
  CKL();
  if (!is_dev) CK(cudaMemcpyAsync(grad, out, 4 * nd, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
}

// Shifting by optimisation: the objective's passes on fresh cells of the current positions, the
// per-scene loss summed into loss_slot (S doubles, zeroed here), the gradient into opt_G, and with
// `out` a descent step into that buffer.
void Scene::opt_passes(const ShiftObjective& o, const Arrays* out, float step, double* loss_slot) {
  if (!opt_S1) {
    opt_S1 = (float4*)mem.get(sizeof(float4) * N);
    opt_S2 = (float4*)mem.get(sizeof(float4) * N);
    opt_XB = (float4*)mem.get(sizeof(float4) * N);
    opt_G = (float4*)mem.get(sizeof(float4) * N);
    opt_V = (float*)mem.get(sizeof(float) * N);
    opt_L = (float*)mem.get(sizeof(float) * N);
  }
  TravArgs t = trav(buf[cur], keys_sorted, cell_off);
  t.pair_count = nullptr;
  prof_begin(7);  // the objective
  if (D == 2) {
    if (kern == 0) launch_opt_forward<2, 0>(t, tiles, d_ntiles, tiles_upper, o, opt_S1, opt_S2, opt_V, opt_L, st);
    else launch_opt_forward<2, 1>(t, tiles, d_ntiles, tiles_upper, o, opt_S1, opt_S2, opt_V, opt_L, st);
  } else {
    if (kern == 0) launch_opt_forward<3, 0>(t, tiles, d_ntiles, tiles_upper, o, opt_S1, opt_S2, opt_V, opt_L, st);
    else launch_opt_forward<3, 1>(t, tiles, d_ntiles, tiles_upper, o, opt_S1, opt_S2, opt_V, opt_L, st);
  }
  CKL();
  prof_end();
  prof_begin(8);  // its gradient (and the descent step)
  if (D == 2) {
    if (kern == 0) launch_opt_backward<2, 0>(t, tiles, d_ntiles, tiles_upper, o, opt_S1, opt_S2, opt_V, opt_XB, opt_G, out, step, st);
    else launch_opt_backward<2, 1>(t, tiles, d_ntiles, tiles_upper, o, opt_S1, opt_S2, opt_V, opt_XB, opt_G, out, step, st);
  } else {
    if (kern == 0) launch_opt_backward<3, 0>(t, tiles, d_ntiles, tiles_upper, o, opt_S1, opt_S2, opt_V, opt_XB, opt_G, out, step, st);
    else launch_opt_backward<3, 1>(t, tiles, d_ntiles, tiles_upper, o, opt_S1, opt_S2, opt_V, opt_XB, opt_G, out, step, st);
  }
  CKL();
  prof_end();
  launches += 5;
  CK(cudaMemsetAsync(loss_slot, 0, sizeof(double) * S, st));
  launch_sum_segments(opt_L, dseg, S, sum_nch, sum_chunk, sum_ctr, loss_slot, st);
  CKL();
  ++launches;
}

static ShiftObjective check_objective(const sph_shift_objective& q) {
  const float w[5] = {q.w_color, q.w_grad, q.w_density, q.w_reg, q.reg_fraction};
  for (float v : w)
    if (!(v >= 0.f) || !std::isfinite(v)) einval("objective weights and reg_fraction must be finite and >= 0");
  if (q.target_kind != 0 && q.target_kind != 1) einval("target_kind must be 0 (sinusoid) or 1 (step)");
  ShiftObjective o;
  o.w_color = q.w_color; o.w_grad = q.w_grad; o.w_density = q.w_density; o.w_reg = q.w_reg;
  o.reg_fraction = q.reg_fraction; o.target_kind = q.target_kind;
  o.t_base = q.t_base; o.t_amp = q.t_amp; o.t_phase = q.t_phase; o.t_lo = q.t_lo; o.t_hi = q.t_hi; o.t_c = q.t_c;
  for (int k = 0; k < 3; ++k) {
    o.t_k[k] = q.t_k[k];
    o.t_n[k] = q.t_n[k];
  }
  return o;
}

void Scene::shift_gradient(const ShiftObjective& o, double* loss, float* grad, int is_dev) {
  for (int s = 0; s < S; ++s)
    if (segs[s].nf < 1) einval("sph_shift_gradient: every scene needs fluid particles");
  host_rebuild();  // cells of the current positions
  if (opt_loss_cap < 1) {
    opt_loss = (double*)mem.get(sizeof(double) * S);
    opt_loss_cap = 1;
  }
  opt_passes(o, nullptr, 0.f, opt_loss);
  if (loss) CK(cudaMemcpyAsync(loss, opt_loss, sizeof(double) * S, cudaMemcpyDeviceToHost, st));
  if (grad) {
    const size_t nd = (size_t)N * D;
    float* outp = is_dev ? grad : (float*)mem_tmp(sizeof(float) * (nd + 64));
    // the adjoint's unpermuting store writes the xyz of a float4 array to original rows
    if (D == 2)
      launch_adj_store<2>(N, buf[cur].meta, d_orig_base, opt_G, opt_G, outp, nullptr, nullptr, st);
    else
      launch_adj_store<3>(N, buf[cur].meta, d_orig_base, opt_G, opt_G, outp, nullptr, nullptr, st);
    CKL();
    if (!is_dev) CK(cudaMemcpyAsync(grad, outp, 4 * nd, cudaMemcpyDeviceToHost, st));
  }
  CK(cudaStreamSynchronize(st));
}

void Scene::shift_descend(const ShiftObjective& o, int n_iters, float step, double* loss_hist) {
  if (n_iters < 1 || !(step >= 0.f) || !std::isfinite(step)) einval("sph_shift_descend: n_iters >= 1 and a finite step >= 0");
  for (int s = 0; s < S; ++s)
    if (segs[s].nf < 1) einval("sph_shift_descend: every scene needs fluid particles");
  if (opt_loss_cap < n_iters) {
    opt_loss = (double*)mem.get(sizeof(double) * (size_t)S * n_iters);
    opt_loss_cap = n_iters;
  }
  for (int it = 0; it < n_iters; ++it) {
    host_rebuild();
    opt_passes(o, &buf[1 - cur], step, opt_loss + (size_t)it * S);
    cur = 1 - cur;
  }
  cells_valid = false;  // the positions moved after the last build
  if (loss_hist) CK(cudaMemcpyAsync(loss_hist, opt_loss, sizeof(double) * S * n_iters, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
}

// Launch and rebuild counters since the scene was created (device rebuilds read back).
void Scene::stats(int64_t* steps, int64_t* rebuilds, int64_t* n_launches) {
  RebuildCtl c{};
  if (d_ctl) {
    CK(cudaMemcpyAsync(&c, d_ctl, sizeof(c), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
  }
  if (steps) *steps = steps_total;
  if (rebuilds) *rebuilds = host_rebuilds + c.rebuilds;
  if (n_launches) *n_launches = launches_total + c.rebuilds * body_launches;
}

void Scene::debug_cells(int64_t* start, int32_t* ids) {
  // the cells of the current positions in the stable order by cell (plain cell keys: the x
  // sub-bins of the 3D sweep's keys are left out, and restored by a rebuild at the next step)
  const bool xo = xorder;
  xorder = false;
  cells_valid = false;
  try {
    ensure_cells();
  } catch (...) {
    xorder = xo;
    throw;
  }
  xorder = xo;
  if (xo) cells_valid = false;
  std::vector<int> off((size_t)C_tot + 1);
  std::vector<uint2> meta(N);
  CK(cudaMemcpyAsync(off.data(), cell_off, sizeof(int) * ((size_t)C_tot + 1), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(meta.data(), buf[cur].meta, sizeof(uint2) * N, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (start)
    for (size_t c = 0; c <= (size_t)C_tot; ++c) start[c] = off[c];
  if (ids)
    for (int k = 0; k < N; ++k) ids[k] = (int32_t)(meta[k].x & ~kWallBit) + orig_base[meta[k].y];
}

// Widen the FP32 guard band of the exact pair predicate to the actual coordinate range (single
// scene); returns the band as an absolute bound on the FP32 error of a squared distance below H^2.
double Scene::pair_band() {
  std::vector<float4> X(N);
  CK(cudaMemcpyAsync(X.data(), buf[cur].X, sizeof(float4) * N, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  double mx = 1.0;
  for (int k = 0; k < N; ++k) {
    float c[3] = {X[k].x, X[k].y, D == 3 ? X[k].z : 0.f};
    for (int q = 0; q < D; ++q) mx = std::max(mx, (double)std::fabs(c[q]));
  }
  for (int q = 0; q < D; ++q) mx = std::max(mx, std::fabs(segs[0].lo_d[q]) + segs[0].L_d[q]);
  DevSeg g = segs[0];
  double H = g.H;
  double band = std::max(1e-5, 4.0 * 8.0 * std::ldexp(mx, -23) / H);
  g.band_lo = (float)(H * H * (1.0 - band));
  g.band_hi = (float)(H * H * (1.0 + band));
  CK(cudaMemcpyAsync(dseg, &g, sizeof(DevSeg), cudaMemcpyHostToDevice, st));
  return band * H * H;
}

// Per-particle support radii (variable support queries): 0 < H_i <= the scene's H, by row.
void Scene::set_support(const float* H, int is_dev) {
  std::vector<float> h((size_t)N);
  CK(cudaMemcpyAsync(h.data(), H, sizeof(float) * N, is_dev ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost, st));
  CK(cudaStreamSynchronize(st));
  for (int s = 0; s < S; ++s)
    for (int k = 0; k < segs[s].p1 - segs[s].p0; ++k) {
      const float v = h[(size_t)orig_base[s] + k];
      if (!(v > 0.f && v <= segs[s].H)) einval("sph_set_support: every H_i must satisfy 0 < H_i <= the scene's H");
    }
  float* d = (float*)mem_tmp(sizeof(float) * ((size_t)N + 64));
  CK(cudaMemcpyAsync(d, h.data(), sizeof(float) * N, cudaMemcpyHostToDevice, st));
  launch_set_support(N, buf[cur].meta, d_orig_base, d, buf[cur].O, st);
  CKL();
  CK(cudaStreamSynchronize(st));
  var_support = true;
}

void Scene::support_query(float* sr, float* rs, float* rg, int is_dev) {
  if (S > 1) einval("sph_support_query supports single scenes");
  if (skin > 0.f) cells_valid = false;
  ensure_cells();
  const double band = pair_band();
  float4* Hs = (float4*)mem_tmp(sizeof(float4) * (2 * (size_t)N + 16) + sizeof(float) * (3 * (size_t)N + 64));
  float4* out = Hs + N;
  float* h = (float*)(out + N + 16);
  TravArgs t = trav(buf[cur], keys_sorted, cell_off);
  t.pair_count = nullptr;
  if (D == 2) {
    if (kern == 0) launch_varsupport<2, 0>(t, tiles, d_ntiles, tiles_upper, Hs, out, (float)band, st);
    else launch_varsupport<2, 1>(t, tiles, d_ntiles, tiles_upper, Hs, out, (float)band, st);
  } else {
    if (kern == 0) launch_varsupport<3, 0>(t, tiles, d_ntiles, tiles_upper, Hs, out, (float)band, st);
    else launch_varsupport<3, 1>(t, tiles, d_ntiles, tiles_upper, Hs, out, (float)band, st);
  }
  CKL();
  float* a = is_dev ? sr : (sr ? h : nullptr);
  float* b = is_dev ? rs : (rs ? h + N : nullptr);
  float* c = is_dev ? rg : (rg ? h + 2 * (size_t)N : nullptr);
  launch_unpermute3(N, buf[cur].meta, d_orig_base, out, a, b, c, st);
  CKL();
  if (!is_dev) {
    if (sr) CK(cudaMemcpyAsync(sr, h, sizeof(float) * N, cudaMemcpyDeviceToHost, st));
    if (rs) CK(cudaMemcpyAsync(rs, h + N, sizeof(float) * N, cudaMemcpyDeviceToHost, st));
    if (rg) CK(cudaMemcpyAsync(rg, h + 2 * (size_t)N, sizeof(float) * N, cudaMemcpyDeviceToHost, st));
  }
  CK(cudaStreamSynchronize(st));
  // the debug band stays widened; restore the scene's own
  CK(cudaMemcpyAsync(dseg, segs.data(), sizeof(DevSeg) * S, cudaMemcpyHostToDevice, st));
}

void Scene::debug_pairs(int64_t* n_pairs, int32_t* pi, int32_t* pj, int64_t cap) {
  if (S > 1) einval("sph_debug_pairs supports single scenes");
  if (skin > 0.f) cells_valid = false;
  ensure_cells();
  pair_band();
  int64_t c = std::max<int64_t>(cap, 0);
  int32_t* dpi = (int32_t*)mem_tmp(sizeof(int32_t) * (2 * (size_t)c + 64));
  int32_t* dpj = dpi + c;
  unsigned long long* cnt = d_pairs + 1;
  CK(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), st));
  TravArgs t = trav(buf[cur], keys_sorted, cell_off);
  t.pair_count = nullptr;
  if (D == 2)
    launch_pairs_t<2>(t, tiles, d_ntiles, tiles_upper, dpi, dpj, cnt, (long long)c, var_support, st);
  else
    launch_pairs_t<3>(t, tiles, d_ntiles, tiles_upper, dpi, dpj, cnt, (long long)c, var_support, st);
  CKL();
  unsigned long long h = 0;
  CK(cudaMemcpyAsync(&h, cnt, sizeof(h), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  *n_pairs = (int64_t)h;
  int64_t w = std::min<int64_t>((int64_t)h, c);
  if (w > 0) {
    CK(cudaMemcpyAsync(pi, dpi, sizeof(int32_t) * w, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(pj, dpj, sizeof(int32_t) * w, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
  }
  CK(cudaMemcpyAsync(dseg, segs.data(), sizeof(DevSeg), cudaMemcpyHostToDevice, st));
}

void Scene::timing(int cls, double* ms, int64_t* count) {
  CK(cudaStreamSynchronize(st));
  double tot = 0.0;
  int64_t c = 0;
  std::vector<ProfEvent> keep;
  for (auto& e : prof_events) {
    if (e.cls == cls) {
      float t = 0.f;
      CK(cudaEventElapsedTime(&t, e.a, e.b));
      tot += t;
      ++c;
      event_pool.push_back(e.a);
      event_pool.push_back(e.b);
    } else {
      keep.push_back(e);
    }
  }
  prof_events.swap(keep);
  *ms = tot;
  *count = c;
}

}  // namespace sph

// ================================================================== C ABI
using sph::Fail;
using sph::Scene;

struct sph_scene {
  Scene s;
};

#define API_BEGIN try {
#define API_END                                     \
  }                                                 \
  catch (const Fail& f) {                           \
    return f.code;                                  \
  }                                                 \
  catch (const std::bad_alloc&) {                   \
    sph::set_err("host allocation failed");         \
    return SPH_ENOMEM;                              \
  }                                                 \
  catch (...) {                                     \
    sph::set_err("unexpected internal exception");  \
    return SPH_EINTERNAL;                           \
  }                                                 \
  return SPH_OK;

extern "C" {

int sph_abi_version(void) { return SPH_ABI_VERSION; }
const char* sph_last_error(void) { return sph::last_error(); }

int sph_set_allocator(sph_alloc_fn a, sph_free_fn f, void* ctx) {
  if ((a == nullptr) != (f == nullptr)) {
    sph::set_err("alloc and free hooks must both be set or both be NULL");
    return SPH_EINVAL;
  }
  sph::set_allocator(a, f, ctx);
  return SPH_OK;
}

static int init_scenes(int S, const sph_params* params, const int* n_fluid, const int* n_wall, const float* const* x,
                       const float* const* v, const float* const* rho, const float* const* mass, int ptr_is_device,
                       void* cuda_stream, sph_scene** out) {
  if (S < 1 || !params || !n_fluid || !n_wall || !x || !rho || !mass || !out) {
    sph::set_err("sph_init: params, counts, x, rho, mass and out must be non-NULL");
    return SPH_EINVAL;
  }
  *out = nullptr;
  sph_scene* sc = nullptr;
  try {
    std::vector<sph_params> prm(params, params + S);
    std::vector<int> nf(n_fluid, n_fluid + S), nw(n_wall, n_wall + S);
    std::vector<double> mx(S, 1.0);
    for (int k = 0; k < S; ++k) {
      if (!x[k] || !rho[k] || !mass[k]) sph::einval("sph_init: missing array of scene " + std::to_string(k));
      for (int q = 0; q < 3; ++q)
        mx[k] = std::max(mx[k], std::max(std::fabs(params[k].box_lo[q]), std::fabs(params[k].box_hi[q])));
      if (!ptr_is_device) {
        const size_t nd = (size_t)(n_fluid[k] + n_wall[k]) * (size_t)std::max(params[k].dim, 1);
        for (size_t q = 0; q < nd; ++q) {
          if (!std::isfinite(x[k][q])) sph::einval("non-finite initial position");
          mx[k] = std::max(mx[k], (double)std::fabs(x[k][q]));
        }
      } else {
        mx[k] = std::max(mx[k], 16.0);
      }
    }
    sc = new sph_scene();
    Scene& s = sc->s;
    sph::init_mem(s.mem);
    s.setup_checked(prm, nf, nw, mx);
    s.bind_stream((cudaStream_t)cuda_stream);
    s.enter();
    s.alloc_all();
    for (int k = 0; k < S; ++k) s.upload(k, x[k], v ? v[k] : nullptr, rho[k], mass[k], ptr_is_device);
    CK(cudaStreamSynchronize(s.st));
    *out = sc;
    sc = nullptr;
  } catch (const Fail& f) {
    delete sc;
    return f.code;
  } catch (...) {
    delete sc;
    sph::set_err("sph_init: unexpected failure");
    return SPH_EINTERNAL;
  }
  return SPH_OK;
}

int sph_init(const sph_params* params, int n_fluid, int n_wall, const float* x, const float* v, const float* rho,
             const float* mass, int ptr_is_device, void* cuda_stream, sph_scene** out) {
  return init_scenes(1, params, &n_fluid, &n_wall, &x, &v, &rho, &mass, ptr_is_device, cuda_stream, out);
}

int sph_init_batch(int n_scenes, const sph_params* params, const int* n_fluid, const int* n_wall,
                   const float* const* x, const float* const* v, const float* const* rho, const float* const* mass,
                   int ptr_is_device, void* cuda_stream, sph_scene** out) {
  return init_scenes(n_scenes, params, n_fluid, n_wall, x, v, rho, mass, ptr_is_device, cuda_stream, out);
}

int sph_batch_info(const sph_scene* sc, int* n_scenes, int32_t* first_row, int32_t* n_rows) {
  if (!sc) {
    sph::set_err("sph_batch_info: NULL scene");
    return SPH_EINVAL;
  }
  if (n_scenes) *n_scenes = sc->s.S;
  for (int k = 0; k < sc->s.S; ++k) {
    if (first_row) first_row[k] = sc->s.orig_base[k];
    if (n_rows) n_rows[k] = sc->s.segs[k].p1 - sc->s.segs[k].p0;
  }
  return SPH_OK;
}

int sph_step(sph_scene* sc, int n_steps) {
  if (!sc || n_steps < 0) {
    sph::set_err("sph_step: bad arguments");
    return SPH_EINVAL;
  }
  API_BEGIN
  sc->s.enter();
  sc->s.tape_valid = false;
  sc->s.steps(n_steps);
  API_END
}

int sph_get_state(const sph_scene* sc, float* x, float* v, float* rho, int ptr_is_device) {
  if (!sc) {
    sph::set_err("sph_get_state: NULL scene");
    return SPH_EINVAL;
  }
  API_BEGIN
  Scene& s = const_cast<Scene&>(sc->s);
  s.enter();
  s.get_state(x, v, rho, ptr_is_device);
  s.leave();
  API_END
}

int sph_rates(sph_scene* sc, float* a, float* drho, float* rho_used, int ptr_is_device) {
  if (!sc) {
    sph::set_err("sph_rates: NULL scene");
    return SPH_EINVAL;
  }
  API_BEGIN
  sc->s.enter();
  sc->s.rates(a, drho, rho_used, ptr_is_device);
  sc->s.leave();
  API_END
}

int sph_shift_gradient(sph_scene* sc, const sph_shift_objective* obj, double* loss, float* grad, int ptr_is_device) {
  if (!sc || !obj) {
    sph::set_err("sph_shift_gradient: NULL scene or objective");
    return SPH_EINVAL;
  }
  API_BEGIN
  const sph::ShiftObjective o = sph::check_objective(*obj);
  sc->s.enter();
  sc->s.shift_gradient(o, loss, grad, ptr_is_device);
  sc->s.leave();
  API_END
}

int sph_shift_descend(sph_scene* sc, const sph_shift_objective* obj, int n_iters, float step, double* loss_hist) {
  if (!sc || !obj) {
    sph::set_err("sph_shift_descend: NULL scene or objective");
    return SPH_EINVAL;
  }
  API_BEGIN
  const sph::ShiftObjective o = sph::check_objective(*obj);
  sc->s.enter();
  sc->s.shift_descend(o, n_iters, step, loss_hist);
  sc->s.leave();
  API_END
}

int sph_debug_bounded_waits(int* gate_status, int* barrier_status) {
  API_BEGIN
  int dev = 0;
  CK(cudaGetDevice(&dev));
  cudaStream_t st = nullptr;
  CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  void* buf = nullptr;
  CK(cudaMalloc(&buf, 64));
  CK(cudaMemsetAsync(buf, 0, 64, st));
  unsigned* words = (unsigned*)buf;   // [0] gate, [1..2] barrier
  int* status = (int*)buf + 8;        // [8] gate status, [9] barrier status
  sph::launch_debug_gate(words, status, st);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = sph::launch_debug_barrier(words + 1, status + 1, st);
  int h[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, status, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(buf);
  cudaStreamDestroy(st);
  CK(e);
  if (gate_status) *gate_status = h[0];
  if (barrier_status) *barrier_status = h[1];
  API_END
}

int sph_set_adjoint_replay(sph_scene* sc, int replay_interval) {
  if (!sc || replay_interval < 0 || replay_interval > 4096) {
    sph::set_err("sph_set_adjoint_replay: NULL scene or interval outside [0, 4096]");
    return SPH_EINVAL;
  }
  sc->s.replay_k_user = replay_interval;
  return SPH_OK;
}

int sph_adjoint_info(sph_scene* sc, int32_t* replay_interval, int64_t* replay_fallbacks) {
  if (!sc) {
    sph::set_err("sph_adjoint_info: NULL scene");
    return SPH_EINVAL;
  }
  if (replay_interval) *replay_interval = sc->s.replay_k;
  if (replay_fallbacks) *replay_fallbacks = sc->s.replay_fallbacks;
  return SPH_OK;
}

int sph_set_support(sph_scene* sc, const float* H, int ptr_is_device) {
  if (!sc || !H) {
    sph::set_err("sph_set_support: NULL scene or radii");
    return SPH_EINVAL;
  }
  API_BEGIN
  sc->s.enter();
  sc->s.set_support(H, ptr_is_device);
  sc->s.leave();
  API_END
}

int sph_support_query(sph_scene* sc, float* search_radius, float* rho_super, float* rho_gather, int ptr_is_device) {
  if (!sc) {
    sph::set_err("sph_support_query: NULL scene");
    return SPH_EINVAL;
  }
  API_BEGIN
  sc->s.enter();
  sc->s.support_query(search_radius, rho_super, rho_gather, ptr_is_device);
  sc->s.leave();
  API_END
}

int sph_set_ghosts(sph_scene* sc, const float* ghost, int ptr_is_device) {
  if (!sc || !ghost) {
    sph::set_err("sph_set_ghosts: NULL scene or ghost array");
    return SPH_EINVAL;
  }
  API_BEGIN
  sc->s.enter();
  sc->s.set_ghosts(ghost, ptr_is_device);
  sc->s.leave();
  API_END
}

int sph_density_gradient(sph_scene* sc, float* grad, int ptr_is_device) {
  if (!sc || !grad) {
    sph::set_err("sph_density_gradient: NULL scene or output");
    return SPH_EINVAL;
  }
  API_BEGIN
  sc->s.enter();
  sc->s.density_gradient(grad, ptr_is_device);
  sc->s.leave();
  API_END
}

int sph_rollout(sph_scene* sc, int n_steps, int ckpt_every) {
  if (!sc) {
    sph::set_err("sph_rollout: NULL scene");
    return SPH_EINVAL;
  }
  API_BEGIN
  sc->s.enter();
  sc->s.rollout(n_steps, ckpt_every);
  API_END
}

int sph_adjoint(sph_scene* sc, const float* xbar_T, const float* vbar_T, const float* rhobar_T, float* xbar_0,
                float* vbar_0, float* rhobar_0, double* nubar, int ptr_is_device) {
  if (!sc) {
    sph::set_err("sph_adjoint: NULL scene");
    return SPH_EINVAL;
  }
  API_BEGIN
  sc->s.enter();
  sc->s.adjoint(xbar_T, vbar_T, rhobar_T, xbar_0, vbar_0, rhobar_0, nubar, ptr_is_device);
  sc->s.leave();
  API_END
}

int sph_scene_info(const sph_scene* sc, int32_t* ncell3, int32_t* n) {
  if (!sc) {
    sph::set_err("sph_scene_info: NULL scene");
    return SPH_EINVAL;
  }
  if (ncell3)
    for (int k = 0; k < 3; ++k) ncell3[k] = sc->s.segs[0].n[k];
  if (n) *n = sc->s.N;
  return SPH_OK;
}

int sph_stats(sph_scene* sc, int64_t* steps, int64_t* rebuilds, int64_t* launches) {
  if (!sc) {
    sph::set_err("sph_stats: NULL scene");
    return SPH_EINVAL;
  }
  API_BEGIN
  sc->s.enter();
  sc->s.stats(steps, rebuilds, launches);
  API_END
}

int sph_debug_cells(sph_scene* sc, int64_t* cell_start, int32_t* sorted_ids) {
  if (!sc) {
    sph::set_err("sph_debug_cells: NULL scene");
    return SPH_EINVAL;
  }
  API_BEGIN
  sc->s.enter();
  sc->s.debug_cells(cell_start, sorted_ids);
  API_END
}

int sph_debug_pairs(sph_scene* sc, int64_t* n_pairs, int32_t* pi, int32_t* pj, int64_t cap) {
  if (!sc || !n_pairs || (cap > 0 && (!pi || !pj))) {
    sph::set_err("sph_debug_pairs: bad arguments");
    return SPH_EINVAL;
  }
  API_BEGIN
  sc->s.enter();
  sc->s.debug_pairs(n_pairs, pi, pj, cap);
  API_END
}

int sph_set_execution(sph_scene* sc, int use_graphs, int graph_chunk) {
  if (!sc || graph_chunk < 1 || graph_chunk > 4096) {
    sph::set_err("sph_set_execution: NULL scene or graph_chunk outside [1, 4096]");
    return SPH_EINVAL;
  }
  sc->s.use_graphs = use_graphs != 0;
  sc->s.graph_chunk = graph_chunk;
  return SPH_OK;
}

int sph_profile(sph_scene* sc, int enable) {
  if (!sc) return SPH_EINVAL;
  sc->s.profiling = enable != 0;
  return SPH_OK;
}

int sph_timing(sph_scene* sc, int cls, double* ms, int64_t* launches) {
  if (!sc || !ms || !launches) return SPH_EINVAL;
  API_BEGIN
  sc->s.timing(cls, ms, launches);
  API_END
}

int sph_counters(sph_scene* sc, int64_t* pairs_per_step, int64_t* launches) {
  if (!sc) return SPH_EINVAL;
  API_BEGIN
  unsigned long long h = 0;
  CK(cudaMemcpyAsync(&h, sc->s.d_pairs, sizeof(h), cudaMemcpyDeviceToHost, sc->s.st));
  CK(cudaStreamSynchronize(sc->s.st));
  if (pairs_per_step) *pairs_per_step = sc->s.last_steps > 0 ? (int64_t)(h / (unsigned long long)sc->s.last_steps) : 0;
  long long cr = 0;
  if (sc->s.dev_policy) {
    CK(cudaMemcpyAsync(&cr, &sc->s.d_ctl->call_rebuilds, sizeof(cr), cudaMemcpyDeviceToHost, sc->s.st));
    CK(cudaStreamSynchronize(sc->s.st));
  }
  if (launches) *launches = sc->s.launches + cr * sc->s.body_launches;
  API_END
}

void sph_destroy(sph_scene* sc) {
  if (!sc) return;
  delete sc;
}

}  // extern "C"
