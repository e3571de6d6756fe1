// gc_launch.h -- host-side launchers of libgcoreccd's kernels (internal).
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "gcoreccd.h"
#include "gc_internal.cuh"

namespace gc {

// Record the text of a failed CUDA call for gc_last_cuda_error and map it to
// a status (GC_ERR_NO_DEVICE, GC_ERR_ALLOC or GC_ERR_CUDA).
gc_status cuda_fail(cudaError_t e);

// j-chunk length of the pair work items for events of the given sizes under
// shape `sh` (R, small_n, small_lanes, n_blocks resident blocks), a multiple
// of `gran` (user > 0 forces it, rounded up to a multiple of gran).
int choose_jchunk(const std::vector<long long> &sizes, const PairShape &sh, int user, int gran);

// Shape of the standalone Eq. 6 evaluation (gc_coulomb_field and its
// allocation-free variant) of one event of n carriers; max_chunks > 0 caps
// the number of j-chunks (the partial-sum capacity).
PairShape field_shape(int precision, int sm_count, long long n, long long max_chunks);

// Pair kernel (Eq. 6): precision 0 = FP64 form, 1 = FP32, 2 = FP32 + Kahan,
// 3 = FP16x2; tile_frames != 0 selects the FP32 forms' tile-frame variant.
// V: the autotuner's kernel variant (see pair_min_blocks).
const void *pair_kernel_ptr(int precision, int R, int newton, int tile_frames, int V = 0);
int pair_kernel_occupancy(int precision, int R, int newton, int tile_frames, int V = 0);
cudaError_t launch_pair(const Dev &d, int precision, int newton, cudaStream_t st);

// One time step after the pair sum: integrate (mobility, drift, diffusion,
// update, collection, binning), compaction of the active list, and the
// single-block bookkeeping that prepares the next step.
cudaError_t launch_integrate(const Dev &d, bool fp64, bool init, int grid, cudaStream_t st);
cudaError_t launch_compact(const Dev &d, bool fp64, int grid, cudaStream_t st);
cudaError_t launch_finalize(const Dev &d, bool init, cudaStream_t st);
// FP32 forms with tile frames: the position shadow for the next step (tile
// frames for large events, the event centroid otherwise) and the FP16x2
// extents.  Without tile frames the compaction writes the shadow.
cudaError_t launch_shadow(const Dev &d, int sm_count, cudaStream_t st);
// Stored charge (Sec. 1): the occupied pixels of each event's image, in
// pixel-index order, as the field sources of the coming integrate.
cudaError_t launch_occupied_pixels(const Dev &d, cudaStream_t st);
// Device-side loop condition of a captured WHILE graph node: continue while
// carriers are active, the step limit is not reached and the last pass made
// progress (so the loop always ends).
cudaError_t launch_loop_cond(const Dev &d, cudaGraphConditionalHandle h, int switch_below,
                             cudaStream_t st);
// Fused small-workload step (FP32 forms without Newton step or tile frames,
// and the FP64 form; no stored charge): the pair kernel that also integrates
// each i-tile as its last j-chunk completes, then one block that compacts and
// does the bookkeeping.
const void *fused_pair_kernel_ptr(int precision, int R);
int fused_pair_occupancy(int precision, int R);
cudaError_t launch_fused_pair(const Dev &d, int precision, int grid, cudaStream_t st);
cudaError_t launch_small_tail(const Dev &d, bool fp64, cudaStream_t st);
// Persistent single-event kernel (one event of at most kFusedMax active holes,
// FP64 form or FP32 forms without FP16x2, Newton step, tile frames or stored
// charge): every step until completion or the step limit in one cooperative
// launch of `grid` blocks (at most se_occupancy(...) per SM), one grid barrier
// per step whose waits give up after limit_s (kErrBarrierTimeout); like every
// step it pauses once at most Ctrl::stop_below holes are active.
const void *se_kernel_ptr(int precision, int R);
int se_occupancy(int precision, int R);
cudaError_t launch_se_loop(const Dev &d, int precision, int grid, double limit_s, cudaStream_t st);
// Cluster-resident single-event kernel (one event of at most 2048 active
// holes, FP32 or FP32 + Kahan): every step until completion or the step limit
// in one launch of one cluster of cluster_ctas_for(n) CTAs; availability
// checks that such a cluster fits.
int cluster_ctas_for(int n);
bool cluster_path_available(int precision, int n);
cudaError_t launch_cluster_event(const Dev &d, int precision, int n, cudaStream_t st);
// Grid-resident single-event kernel (one event of at most 4096 active holes,
// FP32 or FP32 + Kahan): every step until completion or the step limit in one
// cooperative launch of resident_grid(sm_count, n, ctas) CTAs, each owning a fixed
// set of holes, exchanging step-tagged words instead of a grid barrier; its
// waits give up after limit_s (kErrBarrierTimeout).  The words take
// resident_words_bytes() of device memory (Dev::rs_rec).
size_t resident_words_bytes();
int resident_grid(int sm_count, int n, int ctas);
bool resident_path_available(int precision, int n, int sm_count);
cudaError_t launch_resident_event(const Dev &d, int precision, int n, int sm_count, int ctas, double limit_s,
                                  cudaStream_t st);
// Runs a barrier that can never complete on `grid` co-resident blocks; the
// error bits it leaves (kErrBarrierTimeout expected) go to *error_bits.
cudaError_t selftest_barrier_timeout(int grid, double limit_s, int *error_bits, cudaStream_t st);
// Recompute the pair work items from the current active offsets (after the
// pair-kernel shape changes).
cudaError_t launch_build_items(const Dev &d, cudaStream_t st);

// Standalone Eq. 6: FP64 [n][3] device positions -> shadow in slot order.
cudaError_t launch_field_prepare(const Dev &d, const double *xyz, int n, bool fp64,
                                 cudaStream_t st);
// E[i][c] = K * sum of the chunk partials.
cudaError_t launch_field_finish(const Dev &d, int n, double *E, cudaStream_t st);

}  // namespace gc
