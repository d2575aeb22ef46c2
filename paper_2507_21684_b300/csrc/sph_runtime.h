// Host-side scene object of the B300 WCSPH library (internal; the public ABI is include/sph.h).
#pragma once
#include <map>
#include <string>
#include <tuple>
#include <utility>
#include <vector>

#include "sph.h"
#include "sph_passes.cuh"
#include "sph_rebuild.cuh"

namespace sph {

// Errors: internal code throws Fail{status}; the C entry points turn it into the return value.
struct Fail {
  int code;
};
void set_err(const std::string& s);
void einval(const std::string& s);
const char* last_error();
void set_allocator(sph_alloc_fn a, sph_free_fn f, void* ctx);

#define CK(call)                                                                     \
  do {                                                                               \
    cudaError_t _e = (call);                                                         \
    if (_e != cudaSuccess) {                                                         \
      sph::set_err(std::string(#call) + ": " + cudaGetErrorString(_e));              \
      throw sph::Fail{SPH_ECUDA};                                                    \
    }                                                                                \
  } while (0)
#define CKL()                                                                        \
  do {                                                                               \
    cudaError_t _e = cudaGetLastError();                                             \
    if (_e != cudaSuccess) {                                                         \
      sph::set_err(std::string("kernel launch: ") + cudaGetErrorString(_e));         \
      throw sph::Fail{SPH_ECUDA};                                                    \
    }                                                                                \
  } while (0)

// Device memory owned by one scene (allocator hook or cudaMalloc); freed with the scene.
struct DeviceMem {
  sph_alloc_fn afn = nullptr;
  sph_free_fn ffn = nullptr;
  void* actx = nullptr;
  void* fctx = nullptr;
  cudaStream_t stream = nullptr;
  std::vector<std::pair<void*, size_t>> blocks;
  size_t total = 0;
  void* get(size_t bytes);
  void release();
  ~DeviceMem();
};
void init_mem(DeviceMem& m);

struct ProfEvent {
  int cls;
  cudaEvent_t a, b;
};

struct TapeSlot {
  Arrays a;            // sweep input records of one step (sorted order of that step)
  uint32_t* keys;      // sorted cell keys in effect
  uint32_t* perm;      // permutation applied at that step's rebuild (if any)
  int* off;            // cell offsets in effect
  Tile* tiles;         // tile table of that cell structure, and its count
  int* ntiles;
  int* boff;           // sub-bin offsets of the cells ordered by x (3D warp-per-tile sweep), or null
};

struct GraphKey {
  int chunk, cur, since, prof;
  bool operator<(const GraphKey& o) const {
    return std::tie(chunk, cur, since, prof) < std::tie(o.chunk, o.cur, o.since, o.prof);
  }
};

// Event-record nodes of a profiled graph: begin/end of one timed launch.
struct GraphProfNode {
  int cls;
  cudaGraphNode_t a, b;
};

// A scene: one or more packed segments (independent SPH problems) advanced together.
struct Scene {
  DeviceMem mem;
  cudaStream_t st = nullptr;        // stream all work of the scene runs on
  cudaStream_t user_st = nullptr;   // caller's stream (0 = legacy default stream)
  bool own_stream = false;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  int S = 0, D = 2, kern = 0, N = 0, nf_total = 0, C_tot = 0, bits = 0, passes = 0;
  bool summation = false, any_walls = false;
  bool renorm = false;              // renormalised delta-SPH diffusion (continuity mode)
  bool shifting = false;            // particle shifting at the end of each step
  bool mdbc = false;                // mDBC wall treatment (ghost nodes) instead of Shepard's
  float4* ghosts = nullptr;         // mDBC ghost node of each particle row (walls), original order
  bool ghosts_set = false;
  // shifting by optimisation (allocated on first use)
  float4 *opt_S1 = nullptr, *opt_S2 = nullptr, *opt_XB = nullptr, *opt_G = nullptr;
  float *opt_V = nullptr, *opt_L = nullptr;
  double* opt_loss = nullptr;
  int opt_loss_cap = 0;
  float4* gradrho = nullptr;        // <grad rho>^L per particle, sorted order (renorm, or on request)
  float skin = 0.f;
  int interval = 1;
  std::vector<DevSeg> segs;
  std::vector<int> orig_base;
  DevSeg* dseg = nullptr;
  int* d_orig_base = nullptr;
  int* d_fluid_base = nullptr;
  Arrays buf[2];
  int cur = 0;
  uint32_t *kA = nullptr, *vA = nullptr, *kB = nullptr, *vB = nullptr;
  uint32_t* keys_sorted = nullptr;
  uint32_t* perm = nullptr;
  int* cell_off = nullptr;
  // 3D warp-per-tile sweep: the cell keys carry x sub-bins (cell * kXBins + bin), so the sort
  // orders every cell by sub-bin, and the permute writes the sub-bins' offsets (bin_off) beside
  // the cells'; host-launched rebuilds only (scenes with the cooperative rebuild keep plain keys)
  bool xorder = false;
  int* bin_off = nullptr;
  uint32_t* scratch = nullptr;
  // cell-block tiles of the current cell structure
  std::vector<int> line_base_h;
  int* line_base = nullptr;
  int n_lines = 0, tiles_upper = 0;
  Tile* tiles = nullptr;
  int* d_ntiles = nullptr;
  int* d_tile_ctr = nullptr;   // dynamic tile counter (zeroed before each tiled launch)
  int* wall_tiles = nullptr;   // tiles holding a wall particle (wall pass)
  uint4* wall_plans = nullptr;  // plans of the tiles holding walls, and of those holding fluid: the
  uint4* fluid_plans = nullptr; // task lists of the fused wall + sweep launch (TilePlan)
  int* d_nwall = nullptr;      // the two lists' lengths
  int* d_status = nullptr;
  unsigned long long* d_pairs = nullptr;
  double* d_nubar = nullptr;
  double* sum_chunk = nullptr;      // scratch of the per-scene sums (launch_sum_segments)
  int* sum_ctr = nullptr;
  int sum_nch = 1;
  void* tmp = nullptr;
  size_t tmp_bytes = 0;
  bool cells_valid = false;
  int steps_since_build = 0;
  // Verlet skin: the rebuild is decided on the device inside the step graph (conditional node)
  bool dev_policy = false;          // skin large enough for the displacement check
  float inv_r2 = 0.f;               // 1 / (skin/2 - margin)^2
  RebuildCtl* d_ctl = nullptr;
  float4* xbuild = nullptr;         // folded positions at the last build
  float* pairs_pos = nullptr;       // 3D: the sweep input's positions as pairs (warp-per-tile sweep)
  cudaStream_t st_body = nullptr;   // captures the rebuild body of a conditional node
  bool use_coop = false;            // decide in the sweep, rebuild in one cooperative launch
  bool eager_dev = false;           // eager steps also take the device's rebuild decision (the server's batches)
  int coop_grid = 0;
  unsigned* d_bar = nullptr;        // grid barrier of the cooperative rebuild
  bool in_body = false;
  long long body_launches = 0;      // kernels in one conditional rebuild body
  // cumulative counters (since the scene was created)
  long long launches_total = 0, steps_total = 0, host_rebuilds = 0;
  // execution
  bool use_graphs = true;
  int graph_chunk = 8;
  bool capturing = false;
  std::map<GraphKey, cudaGraphExec_t> graphs;
  std::map<GraphKey, long long> graph_launch_count;
  std::map<GraphKey, std::vector<GraphProfNode>> graph_prof;
  std::vector<cudaGraph_t> graph_templates;  // kept alive: profiled graphs address their nodes
  std::vector<ProfEvent> capture_events;   // events recorded while capturing (profiling)
  std::vector<cudaEvent_t> event_pool;
  cudaEvent_t take_event();
  // profiling and counters
  bool profiling = false;
  std::vector<ProfEvent> prof_events;
  long long launches = 0;
  int last_steps = 0;
  // adjoint tape
  bool tape_valid = false;
  int tape_n = 0, tape_k = 0, tape_cap = 0;
  std::vector<Arrays> ckpts;
  // two tapes: the replay of a segment fills one while the reverse pass of the segment after it
  // reads the other (the replay runs on st_rep, the reverse pass on st)
  std::vector<TapeSlot> tapes[2];
  bool adj_alloc = false;
  float4* XB[2] = {nullptr, nullptr};
  float4* VB[2] = {nullptr, nullptr};
  float4* Sd = nullptr;
  float* Pp = nullptr;
  double* nu_acc = nullptr;         // adjoint: per storage slot, the viscosity adjoint summed over the steps
  Arrays scratch_arr{};
  Arrays rep_out[2]{};               // a replay's sweep output before a rebuild, per tape ([0] is scratch_arr)
  int* d_tile_ctr_b = nullptr;      // tile counter of the reverse pass's launches (beside the replay's)
  cudaStream_t st_rep = nullptr;    // the adjoint's forward replays
  cudaEvent_t ev_rep[2] = {nullptr, nullptr};   // a tape's replay finished
  cudaEvent_t ev_free[2] = {nullptr, nullptr};  // a tape's reverse pass finished (the tape is free)
  Arrays ckpt_work{};               // the segment's checkpoint, copied (graphs do not depend on it)
  std::map<long long, std::pair<cudaGraphExec_t, long long>> adj_graphs;  // by part, tape, interval, length
  int replay_k = 1;                 // rebuild interval of the adjoint's forward replay (skin > 0)
  int replay_k_user = 0;            // the caller's interval (0: from the rollout's rebuild rate)
  int* d_replay_flag = nullptr;     // [0] a replayed step outgrew the skin, [1] scratch
  float* adj_rows = nullptr;        // the running adjoint by original row (segment boundaries)
  unsigned* d_replay_maxr = nullptr;
  long long replay_fallbacks = 0;

  ~Scene();
  void bind_stream(cudaStream_t user);
  void enter();
  void leave();
  void setup_checked(const std::vector<sph_params>& prms, const std::vector<int>& nfs,
                     const std::vector<int>& nws, const std::vector<double>& max_abs_x);
  void alloc_all();
  void alloc_arrays(Arrays& a);
  void copy_arrays(const Arrays& dst, const Arrays& src);
  void upload(int s, const float* x, const float* v, const float* rho, const float* mass, int is_dev);
  void* mem_tmp(size_t bytes);
  TravArgs trav(const Arrays& a, const uint32_t* keys, const int* off, const int* boff = nullptr) const;
  void prof_begin(int cls);
  void prof_end();
  std::pair<uint32_t*, uint32_t*> rebuild(const Arrays& in, const Arrays& out, uint32_t* keys_out,
                                          uint32_t* perm_out, int* off_out, Tile* tiles_out = nullptr,
                                          int* ntiles_out = nullptr, int* boff_out = nullptr);
  void build_tiles(const int* off, const uint2* meta, Tile* tl, int* ntl);
  bool fuse_walls = true;           // wall pass inside the sweep launch (Shepard walls, MC diffusion;
                                    // in summation mode after the density launch)
  bool walls_in_sweep() const { return fuse_walls && any_walls && !renorm && !mdbc; }
  // fused_walls: the sweep launch does the wall pass (walls_in_sweep()), so it is left out here
  void passes_before_sweep(const TravArgs& t, const Tile* tl = nullptr, const int* ntl = nullptr,
                           bool fused_walls = false);
  void walls_pass(const TravArgs& t, const Tile* tl);
  void set_ghosts(const float* g, int is_dev);
  bool var_support = false;         // per-particle support radii set (the records' H_i)
  double pair_band();
  void set_support(const float* H, int is_dev);
  void support_query(float* sr, float* rs, float* rg, int is_dev);
  void need_ghosts() const;
  void grad_pass(const TravArgs& t, const Tile* tl, const int* ntl);
  void sweep(const TravArgs& t, const Arrays& out, const Tile* tl = nullptr, const int* ntl = nullptr,
             bool fused_walls = false, const Displace* disp = nullptr);
  void host_rebuild();
  void step_once();
  void step_conditional();
  void step_coop();
  void cond_rebuild(int count);
  void coop_rebuild();
  void shift_pass();
  RebuildArgs coop_args(const Arrays& in, const Arrays& out, int* off, const int* flag, int copy_back);
  void advance_schedule();
  void steps(int n);
  void ensure_cells();
  void rollout(int n, int k);
  void alloc_tape(int k);
  void adjoint_replay(int L, int K, int b);
  void adjoint_backward(int L, int K, int b);
  void adjoint_part(int part, int L, int K, int b);
  int adjoint_replay_segment(int sgi, int b);
  void adjoint(const float* xb, const float* vb, const float* rb, float* xb0, float* vb0, float* rb0, double* nub,
               int is_dev);
  void get_state(float* x, float* v, float* rho, int is_dev);
  void check_status();
  std::vector<int> status_words();
  void clear_unstable();
  void rates(float* a, float* drho, float* rho, int is_dev);
  void density_gradient(float* grad, int is_dev);
  void opt_passes(const ShiftObjective& o, const Arrays* out, float step, double* loss_slot);
  void shift_gradient(const ShiftObjective& o, double* loss, float* grad, int is_dev);
  void shift_descend(const ShiftObjective& o, int n_iters, float step, double* loss_hist);
  void debug_cells(int64_t* start, int32_t* ids);
  void debug_pairs(int64_t* n_pairs, int32_t* pi, int32_t* pj, int64_t cap);
  void timing(int cls, double* ms, int64_t* count);
  void stats(int64_t* steps, int64_t* rebuilds, int64_t* launches);
};

// device bytes of a scene's wall-task lists (fused wall + sweep launch), as alloc_all sizes them
size_t wall_plan_bytes(const sph_params& p, int n_fluid, int n);

}  // namespace sph
