// Launch interface of the tiled neighbour passes (host side of sph_passes.cu).
#pragma once
#include "sph_kernels.cuh"
#include "sph_tiles.cuh"

namespace sph {

cudaError_t configure_passes();
// kernels one sweep launch call issues (the 3D warp-per-tile sweep packs the positions first)
int sweep_kernels(int dim, long long N, const float* packed);
// Floats of the 3D sweep's scratch of positions as pairs (TravArgs::packed) for N particles.
size_t packed_pairs_floats(long long N);
// Whether the sweep of a scene of this dimension and size runs on the warp-per-tile traversal.
bool warp_sweep(int dim, long long N);
void launch_debug_gate(const unsigned* gate, int* status, cudaStream_t st);
template <int D>
void launch_tiles(const DevSeg* segs, int S, const int* line_base, int n_lines, const int* cell_off, Tile* tiles,
                  int* ntiles, cudaStream_t st);
template <int D, int KERN>
void launch_walls_t(const TravArgs& t, const Tile* tiles, const int* wall_tiles, const int* n_wall_tiles,
                    int tiles_upper, cudaStream_t st);
// tiles holding walls into list (indices) and wall_p (plans), tiles holding fluid into fluid_p
// (plans), the two counts into count[0..1]
template <int D>
void launch_wall_tiles(const Tile* tiles, const int* ntiles, int tiles_upper, const uint2* meta, int* list,
                       uint4* wall_p, uint4* fluid_p, int* count, cudaStream_t st);
template <int D, int KERN>
void launch_density_t(const TravArgs& t, const Tile* tiles, const int* ntiles, int tiles_upper, cudaStream_t st);
template <int D, int KERN>
void launch_mdbc(const TravArgs& t, const Tile* tiles, const int* wall_tiles, const int* n_wall_tiles, int tiles_upper,
                 const float4* ghost, const int* orig_base, cudaStream_t st);
// wall tasks from wall_p, sweep tasks from fluid_p (tile plans, TilePlan<D>::U4 words each;
// lengths n_lists[0], n_lists[1]); the launch fills in the plans' staging tables
template <int D, int KERN>
void launch_walls_sweep_t(const TravArgs& t, uint4* wall_p, uint4* fluid_p, const int* n_lists,
                          int tiles_upper, const Arrays& out, const Displace& disp, cudaStream_t st);
template <int D, int KERN>
void launch_grad_t(const TravArgs& t, const Tile* tiles, const int* ntiles, int tiles_upper, float4* grad,
                   cudaStream_t st);
// grad != nullptr selects the renormalised diffusion (gradients from launch_grad_t)
template <int D, int KERN>
void launch_sweep_t(const TravArgs& t, const Tile* tiles, const int* ntiles, int tiles_upper, const Arrays& out,
                    const Displace& disp, const float4* grad, cudaStream_t st);
template <int D, int KERN>
void launch_rates_t(const TravArgs& t, const Tile* tiles, const int* ntiles, int tiles_upper, const RateOut& ro,
                    const float4* grad, cudaStream_t st);
template <int D, int KERN>
void launch_shift_t(const TravArgs& t, const Tile* tiles, const int* ntiles, int tiles_upper, const Arrays& out,
                    const Displace& disp, cudaStream_t st);
template <int D, int KERN>
void launch_opt_forward(const TravArgs& t, const Tile* tiles, const int* ntiles, int tiles_upper,
                        const ShiftObjective& o, float4* S1, float4* S2, float* V, float* Lp, cudaStream_t st);
template <int D, int KERN>
void launch_opt_backward(const TravArgs& t, const Tile* tiles, const int* ntiles, int tiles_upper,
                         const ShiftObjective& o, const float4* S1, const float4* S2, const float* V, float4* XB,
                         float4* G, const Arrays* out, float step, cudaStream_t st);
template <int D>
void launch_pairs_t(const TravArgs& t, const Tile* tiles, const int* ntiles, int tiles_upper, int32_t* pi, int32_t* pj,
                    unsigned long long* count, long long cap, bool var, cudaStream_t st);
template <int D, int KERN>
void launch_varsupport(const TravArgs& t, const Tile* tiles, const int* ntiles, int tiles_upper, float4* Hs,
                       float4* out, float band, cudaStream_t st);
void launch_set_support(int N, const uint2* meta, const int* orig_base, const float* H, float4* O, cudaStream_t st);
void launch_unpermute3(int N, const uint2* meta, const int* orig_base, const float4* src, float* a, float* b, float* c,
                       cudaStream_t st);
template <int D, int KERN>
void launch_adj_t(const TravArgs& t, const Tile* tiles, const int* ntiles, int tiles_upper, const float4* S,
                  const float* Pp, const float4* XBin, const float4* VBin, float4* XBout, float4* VBout,
                  double* nu_acc, cudaStream_t st);
// summation mode: the adjoint of rho^ = sum_j m_j W_ij (left in XBin.w) passed to the positions
template <int D, int KERN>
void launch_adj_dens_t(const TravArgs& t, const Tile* tiles, const int* ntiles, int tiles_upper, const float4* XBin,
                       const float4* VBin, float4* XBout, float4* VBout, cudaStream_t st);
void launch_sum_float_partials(const float* part, int n, double* acc, cudaStream_t st);
// Per-scene FP64 sums of per-particle partials; chunk: S x nchunks doubles, ctr: S ints (zeroed
// once, left zeroed), nchunks = sum_segments_chunks(largest scene's particle count).
int sum_segments_chunks(long long max_seg_n);
void launch_sum_segments(const float* part, const DevSeg* segs, int S, int nchunks, double* chunk, int* ctr,
                         double* acc, cudaStream_t st);
void launch_sum_segments(const double* part, const DevSeg* segs, int S, int nchunks, double* chunk, int* ctr,
                         double* acc, cudaStream_t st);

}  // namespace sph
