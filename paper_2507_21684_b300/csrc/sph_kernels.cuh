// Launch interface of the element-wise and sorting kernels (host side of sph_kernels.cu).
#pragma once
#include "sph_device.cuh"

namespace sph {

// Arguments shared by every neighbour pass.
struct TravArgs {
  const DevSeg* segs;
  int N;
  Arrays a;                  // current (sorted) particle arrays
  const uint32_t* keys;      // sorted global cell key per particle
  const int* cell_off;       // CSR offsets over global cells
  int* status;               // device error word (bit 0: unstable state)
  unsigned long long* pair_count;  // optional: in-radius pairs of fluid particles
  int* tile_ctr;             // [0] dynamic tile counter, [1] finished CTAs (both zero between launches)
  float* packed;             // 3D: scratch of the positions as pairs for the warp-per-tile sweep (or null)
  const int* bin_off;        // 3D: CSR offsets over cell * kXBins + x sub-bin (keys with sub-bins), or null
  int kshift;                // keys >> kshift is the cell key (kXShift when the keys carry x sub-bins)
};

// Device-side rebuild policy state of a scene (Verlet skin).
struct RebuildCtl {
  int since;             // sweeps served by the current cell structure
  unsigned maxr;         // max over fluid of |x - x_build|^2 / (skin/2 - margin)^2 (float bits)
  long long rebuilds;    // device-decided rebuilds taken (cumulative)
  long long call_rebuilds;  // device-decided rebuilds since the host last zeroed it (one API call)
  int flag;              // the next step rebuilds (set by the sweep's last CTA)
  int pad;
};

// Displacement check written by the sweep's epilogue (all null: no check).
struct Displace {
  const float4* xb;      // folded positions at the last build (x, y[, z], 0)
  unsigned* maxr;        // running maximum (float bits, non-negative)
  float inv_r2;          // 1 / (skin/2 - margin)^2
  RebuildCtl* ctl;       // set: the sweep's last CTA decides the next step's rebuild
  int interval;          // rebuild_interval
  int* sticky;           // set (adjoint replay): the last CTA sets *sticky if the maximum exceeds 1,
                         // then zeroes the maximum
};

// Objective of the shifting-by-optimisation passes (weights, pair penalty, target density).
struct ShiftObjective {
  float w_color, w_grad, w_density, w_reg, reg_fraction;
  int target_kind;  // 0: t_base + t_amp sin(t_k . x + t_phase); 1: t_lo where t_n . x < t_c, else t_hi
  float t_base, t_amp, t_k[3], t_phase;
  float t_lo, t_hi, t_n[3], t_c;
};

// Outputs of the rate evaluation (original order, fluid only).
struct RateOut {
  float* a;
  float* drho;
  float* rho;
  const int* orig_base;      // first fluid row of each scene in the outputs
};

int sort_scratch_words(int N);
void launch_exclusive_scan(uint32_t* a, int n, uint32_t* sums, cudaStream_t st);
// One pass of the radix sort; segs set: the first pass, whose keys come from the state (cell keys,
// with xbins the keys with x sub-bins, cell * kXBins + bin).
template <int D>
void launch_sort_pass(const uint32_t* kin, const uint32_t* vin, uint32_t* kout, uint32_t* vout, int N, int shift,
                      uint32_t* hist, uint32_t* sums, const DevSeg* segs, const Arrays& a, cudaStream_t st,
                      bool xbins = false);
// boff set: the keys carry x sub-bins; off gets the cells' offsets (keys >> kXShift) and boff the
// offsets over cell * kXBins + bin (C * kXBins + 1 entries).
template <int D>
void launch_permute(const DevSeg* segs, int N, const uint32_t* perm, const Arrays& in, const Arrays& out,
                    const uint32_t* keys, int C, int* off, float4* xb, cudaStream_t st, int* boff = nullptr);
template <int D>
void launch_copy_state(int N, const Arrays& src, const Arrays& dst, cudaStream_t st);

// count: 1 when a sweep follows and uses the cells (it counts towards rebuild_interval), else 0
void launch_rebuild_decide(RebuildCtl* ctl, int interval, int count, cudaGraphConditionalHandle h, cudaStream_t st);
template <int D>
void launch_upload(const DevSeg* segs, int seg, int n, int nf, int p0, const float* x, const float* v,
                   const float* rho, const float* mass, const Arrays& a, cudaStream_t st);
template <int D>
void launch_download(int N, const Arrays& a, const int* orig_base, float* x, float* v, float* rho, cudaStream_t st);
template <int D>
void launch_adj_seed(const DevSeg* segs, int N, const Arrays& fw, const float4* XB, const float4* VB, float4* S,
                     float* Pp, cudaStream_t st);
void launch_adj_unpermute(int N, const uint32_t* perm, const float4* XBin, const float4* VBin, float4* XBout,
                          float4* VBout, cudaStream_t st);
template <int D>
void launch_adj_load(int N, const uint2* meta, const int* orig_base, const float* xb, const float* vb,
                     const float* rb, float4* XB, float4* VB, cudaStream_t st);
template <int D>
void launch_adj_store(int N, const uint2* meta, const int* orig_base, const float4* XB, const float4* VB, float* xb,
                      float* vb, float* rb, cudaStream_t st);

template <int D>
void launch_copy_range(const Arrays& src, int s0, const Arrays& dst, int d0, int n, int seg, cudaStream_t st);
template <int D>
void launch_download_range(const Arrays& a, int p0, int n, float* x, float* v, float* rho, cudaStream_t st);

}  // namespace sph
