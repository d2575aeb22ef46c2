/* sph_noalloc.h — cell binning that allocates nothing (libsph_b300.so).
 *
 * The paper has no counterpart to this call: it is a library service, not part of the method.
 * It bins particles into the cells a scene would use (cell key of every particle, stable sort
 * by key, CSR cell ranges) for a caller that must not allocate device memory, and returns the
 * cell structure instead of advancing a scene.
 *
 * Who cannot allocate, and why:
 *   - code that runs inside a device-memory allocator (for example an allocator callback
 *     registered with sph_set_allocator, or a caching allocator's out-of-memory handler):
 *     allocating there re-enters the allocator, which deadlocks on its lock or recurses;
 *   - a process that has handed all free HBM to another pool (a serving loop's reservation)
 *     and must not grow its footprint by even one block;
 *   - latency-critical host threads, for which cudaMalloc / cudaFree are ruled out because
 *     they may synchronise the device.
 * sph_init and the other scene calls allocate (from the sph_set_allocator hook, default the
 * stream-ordered pool); this call only enqueues kernels on the caller's stream.
 *
 * Scratch: one statically sized device array inside the library, SPH_NOALLOC_SCRATCH_BYTES
 * per device (about 6.3 MiB), allocated by the CUDA driver when the library's module is loaded,
 * never by this call.  Limits that follow from it:
 *   n <= SPH_NOALLOC_MAX_PARTICLES (524288); larger n returns SPH_EINVAL with a message.
 * Nothing in the scratch has to start at zero: every word a call reads was written earlier in
 * the same call.
 *
 * Setup: the first call on a device (the device current at the call) looks up the scratch's
 * device address with cudaGetSymbolAddress and keeps it for later calls on that device; it may
 * also make the driver load the library's module.  Make that first call outside any CUDA
 * stream capture (a call with n = 0 is enough).  Later calls do no setup.
 *
 * Concurrency: all calls on one device share the one scratch array.  Two calls whose work
 * overlaps on the device (different streams, or different host threads without ordering)
 * race on it and give wrong results.  Order them: the same stream, or an event between them.
 */
#ifndef SPH_B300_NOALLOC_H
#define SPH_B300_NOALLOC_H
#include "sph.h"

#ifdef __cplusplus
extern "C" {
#endif

#define SPH_NOALLOC_MAX_PARTICLES 524288
#define SPH_NOALLOC_SCRATCH_BYTES (4 * (3 * 524288 + 256 * 256 + 4096))

/* Cell structure of n particles of one scene, without allocating.
 *   params      scene parameters (host); only dim, kernel, box_lo/box_hi, periodic_mask, H and
 *               skin shape the grid (cell edge >= H + skin per axis, as sph_init builds it),
 *               but every field is validated as by sph_init.
 *   x           device pointer, n * dim floats, original particle order (fluid then walls).
 *               Periodic axes are wrapped into the box; other coordinates are clamped to the
 *               edge cells.
 *   n           particle count, 0 <= n <= SPH_NOALLOC_MAX_PARTICLES.
 *   cell_start  device pointer, cell_start_len int32 entries; receives the CSR offsets
 *               cell_start[c] = first sorted position of cell c, for c = 0 .. n_cells
 *               (cell index (cz * ny + cy) * nx + cx).  SPH_EINVAL if cell_start_len < n_cells + 1.
 *   sorted_ids  device pointer to at least n int32 (the call cannot check its length: a shorter
 *               buffer is written past its end); receives the original index of each particle
 *               in cell order, ties in ascending original index (a stable sort).  The sort also
 *               uses it as one of its two value buffers while it runs.
 *   n_cells     host pointer or NULL; receives the number of cells (also on SPH_EINVAL for a
 *               short cell_start, so that a caller can size the buffer and call again).
 *   stream      cudaStream_t of the caller (NULL = legacy default stream).  The call only
 *               enqueues work: outputs are ready when the stream reaches that point.
 * Results equal sph_debug_cells of a freshly initialised scene with the same particles.
 * The caller owns every buffer.  Returns SPH_OK, SPH_EINVAL (bad arguments; nothing enqueued)
 * or SPH_ECUDA (setup or launch failure; sph_last_error says which). */
SPH_API int sph_cells_noalloc(const sph_params* params, const float* x, int32_t n, int32_t* cell_start,
                              int64_t cell_start_len, int32_t* sorted_ids, int32_t* n_cells, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SPH_B300_NOALLOC_H */
