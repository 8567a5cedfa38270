// Device-side planning of a batch whose offsets are in device memory
// (device_plan.cu): the host decides only what does not depend on the
// lengths; the kernels it enqueues do the rest on the stream.
#pragma once

#include <string>

#include "sw_internal.h"

namespace swgb {

// What the host decides before enqueueing: the two arithmetic routes of the
// batched kernel (0: packed 16-bit, 1: scaled int32) and their limits, the
// grids, the bulk lane-group width and cap, the slot size.  Passed to the
// planning kernels by value.
struct DevicePlanShape {
    int32_t n_pairs;
    int32_t A, go, ge;
    int32_t linear, all_plain, ends_only;
    int32_t route_on[2];    // the route's kernel fits the device
    int32_t kind[2];        // ProfileKind of the route's kernel
    int32_t rows[2];        // rows per lane
    int32_t lim[2];         // a pair takes the route when min(n, m) <= lim
    int32_t grid[2], n_warps[2];
    int32_t half_tails[2];  // bulk pairs with a half-used last strip take G / 2
    int32_t bulk_log2g;
    double cap_fraction;
    int32_t strip_ov;       // planner charge per strip start, in steps of the warp
    int32_t slot_words;     // strip-boundary words per lane of a group slot
    int32_t plain_grid;     // blocks of the plain kernel's launches
    int64_t scratch_words;  // slot words of the larger grid
    int32_t guards;         // guard regions around every workspace part (test aid)
    int8_t mat[kMaxAlphabet * kMaxAlphabet];
};

// Fills *out from the host-known arguments (queries the group kernels'
// occupancy on the current device).  Arguments must already be checked.
// min_pairs_per_warp: the grid gets at most one warp per this many pairs
// (1: lowest latency; more: leave room for other launches on the GPU).
int device_plan_shape(int32_t n_pairs, const int8_t *mat, int32_t A, int32_t go, int32_t ge,
                      int32_t mode, int sm_count, int narrow_log2g, double cap_fraction,
                      int slot_words, DevicePlanShape *out, std::string *msg,
                      int min_pairs_per_warp = 1);

// Device bytes of the planning workspace (tables, sort buffers, slots).
size_t device_plan_workspace_bytes(const DevicePlanShape &S);

// Enqueues planning and alignment on s: workspace (256-byte aligned, at
// least device_plan_workspace_bytes) is used for the call's duration on s.
// Pair i's sequences are q[qo[i] .. qo[i + 1]) and r[ro[i] .. ro[i + 1])
// (CSR), or q[qo[i] .. qe[i]) and r[ro[i] .. re[i]) when qe and re are given
// (pairs gathered from anywhere in q and r).
cudaError_t enqueue_device_plan(const DevicePlanShape &S, void *workspace, const int64_t *qo,
                                const int64_t *ro, const uint8_t *q, const uint8_t *r,
                                const Outputs &o, int32_t *status, cudaStream_t s,
                                const int64_t *qe = nullptr, const int64_t *re = nullptr);

// Strip-boundary words per lane of the one-shot call's group slots: a group
// of G lanes holds the boundary rows of sequences up to about 514 G
// residues (longer pairs take wider groups, beyond 32 lanes the plain
// kernel).
constexpr int kOneShotSlotWords = 1028;

}  // namespace swgb
