// Single-launch rebuild of the cell structure (sph_rebuild.cu).
#pragma once
#include "sph_kernels.cuh"
#include "sph_tiles.cuh"

namespace sph {

struct RebuildArgs {
  const DevSeg* segs;
  int S, N, C, passes, nb;         // scenes, particles, cells, radix passes, 2048-key sort tiles
  Arrays in, out;                  // sorted from `in` into `out` (then copied back if copy_back)
  int copy_back;
  uint32_t *kA, *vA, *kB, *vB;     // sort ping-pong buffers (result in kA/vA after an even count)
  uint32_t *hist, *sums;           // 256 x nb digit counts, scan block totals (>= grid words)
  int* off;                        // CSR cell offsets (C + 1)
  int* boff;                       // 3D: keys with x sub-bins; their CSR offsets (C * kXBins + 1), or null
  float4* xb;                      // folded positions at the build (or null)
  const int* line_base;
  int n_lines;
  Tile* tiles;
  int* ntiles;
  int* wall_list;                  // tiles holding walls (or null)
  uint4* wall_plans;               // plans of the tiles holding walls (with wall_list)
  uint4* fluid_plans;              // plans of the tiles holding fluid (with wall_list)
  int* nwall;                      // the two lists' lengths
  const int* flag;                 // rebuild only when *flag != 0 (null: always)
  RebuildCtl* ctl;                 // rebuild counters (or null)
  unsigned* bar;                   // grid barrier words (two, zero at rest)
  int* status;                     // bit 1: a barrier gave up waiting
};

// Grid for the cooperative launch (0 when it cannot be determined).
template <int D>
int rebuild_coop_grid();
template <int D>
cudaError_t launch_rebuild_coop(const RebuildArgs& r, int grid, cudaStream_t st);
// test hook: a two-CTA cooperative launch whose grid barrier one CTA never reaches
cudaError_t launch_debug_barrier(unsigned* bar, int* status, cudaStream_t st);

}  // namespace sph
