// Internal declarations shared by the host API and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

struct sw_ctx;  // the library context (include/swgb.h)

namespace swgb {

// Scores on the batched path are held scaled by 2^16 so that the low half
// of every H value is free for the column part of the end-cell key
// (H << 16) | (65535 - j); one max-plus instruction per cell then tracks the
// maximal cell with the end rule (largest H, then smallest column).
constexpr int kKeyShift = 16;
constexpr int32_t kScaledNegInf = -(1 << 30);  // E/F "-infinity", scaled domain
constexpr int32_t kPlainNegInf = -(1 << 30);   // E/F "-infinity", plain int32
constexpr int32_t kScaledPad = -(1 << 29);     // profile score of rows beyond n
constexpr int kMaxScaledScore = 32766;         // (S << 16) + 65535 < 2^31
// Column part of the end-cell key: kColBase - j.  A lane's last row starts
// up to 2 x 32 - 1 = 63 columns early (pad columns, j >= -63, with split
// rows), so sequences of the batched path are limited to kColBase residues
// to keep the part in [0, 65535).
constexpr int kColBase = 65535 - 64;
constexpr int kMaxScaledGap = 16383;
constexpr int kMaxAlphabet = 32;
#ifndef SWGB_ROWS
#define SWGB_ROWS 16
#endif
constexpr int kRows = SWGB_ROWS;               // query rows per lane (group kernel): 8 or 16
constexpr int kGroupWarps = 4;                 // warps per block (group kernel)
#ifndef SWGB_GROUP_MIN_BLOCKS
#define SWGB_GROUP_MIN_BLOCKS 3
#endif
constexpr int kGroupMinBlocks = SWGB_GROUP_MIN_BLOCKS;  // resident blocks per SM (register cap)
constexpr int kPlainWideThreads = 256;         // plain kernel block for queries > 1024
constexpr int kPlainMaxRows = 256;             // rows per thread there (n <= 65536)

// One pair as the device sees it (plan order).
struct PairInfo {
    int64_t q;        // offset of the first query residue
    int64_t r;        // offset of the first reference residue
    int64_t scratch;  // offset (uint32 units) of the pair's boundary words, or -1
                      // (used only when the launch has no per-group slots)
    int32_t n, m;     // lengths
    int32_t id;       // output position in the caller's batch
    int32_t pad;
};

// A queue of the persistent kernel: `count` consecutive pairs of the plan's
// pair array starting at `first` (sorted by cost, largest first), each
// aligned by a group of G = 1 << log2g lanes.
struct ClassInfo {
    int32_t first;
    int32_t count;
    int32_t log2g;
    int32_t warp_begin;  // warps [warp_begin, next class's warp_begin) start here
};
constexpr int kMaxClasses = 6;  // G = 32, 16, 8, 4, 2 (1 unused)
constexpr int kMinLog2G = 1;    // narrowest lane group: 2 lanes, 16 groups per warp

struct Outputs {
    int32_t *score, *qend, *rend, *qstart, *rstart;
};

struct GroupParams {
    const uint8_t *q;
    const uint8_t *r;
    const PairInfo *pairs;
    const ClassInfo *classes;
    int32_t n_classes;
    int32_t *counters;  // queue heads, one per class, zeroed before each launch
    int32_t n_warps;    // warps of the launch (grid x warps per block)
    uint32_t *scratch;  // strip-boundary words
    // Strip-boundary words per lane of each lane group's own slot (a multiple
    // of 4): the group of lanes [b, b + G) of warp w owns words
    // [(32 w + b) s, (32 w + b + G) s) and reuses them for each pair it
    // aligns.  0: each pair has its own words at PairInfo::scratch.
    int32_t slot_words;
    int32_t *status;    // device status word (0 = ok)
    Outputs out;
    int32_t alphabet;
    int32_t gap_open, gap_extend;  // unscaled, <= 0
    int32_t ends_only;             // skip the reverse pass (qstart/rstart not written)
    int8_t mat[kMaxAlphabet * kMaxAlphabet];
};

struct PlainParams {
    const uint8_t *q;
    const uint8_t *r;
    const PairInfo *pairs;  // one block per entry
    int32_t n_pairs;
    // NULL: pairs[0 .. n_pairs), one per block.  Otherwise the device pair
    // {first, count}: pairs[first .. first + count), taken by the blocks of
    // the grid in turn (the count is known only on the device).
    const int32_t *range;
    int32_t *status;
    Outputs out;
    int32_t alphabet;
    int32_t gap_open, gap_extend;
    int32_t ends_only;
    int8_t mat[kMaxAlphabet * kMaxAlphabet];
};

// Strip-boundary words of a sweep over `cols` columns whose rows span more
// than one strip: two buffers (previous strip's last row / this strip's
// last row) of cols rounded up to a multiple of 4 words, 16-byte aligned,
// plus 4 words of tail so that a 16-byte chunk read past the last column
// stays inside.
inline int64_t boundary_words(int cols) { return 2 * (int64_t)((cols + 3) & ~3) + 4; }

// Scratch words of a batched-path pair on lane groups of G lanes.  The
// forward sweep has the query as rows and the reference as columns; the
// reverse sweep is transposed (reversed reference prefix as rows, reversed
// query prefix as columns), so either may need strips; one buffer sized for
// the longer sequence serves both, one after the other.
inline int64_t pair_scratch_words(int n, int m, int G, int rows_per_lane) {
    const int strip = G * rows_per_lane;
    if (n <= strip && m <= strip) return 0;
    return boundary_words(n > m ? n : m);
}

// Words per lane that a G-lane group's slot needs for a pair (0 when the
// pair fits one strip in both sweeps), rounded up to whole 16-byte chunks.
inline int32_t pair_slot_words(int n, int m, int G, int rows_per_lane) {
    const int64_t w = pair_scratch_words(n, m, G, rows_per_lane);
    return (int32_t)(((w + G - 1) / G + 3) & ~(int64_t)3);
}

// Whether a pair can take the batched kernel's scaled int32 arithmetic.
// Both sweeps index columns below kColBase (the forward one the reference,
// the transposed reverse one the query).
inline bool group_path_eligible(int n, int m, int smax, int gap_open, int gap_extend) {
    if (-gap_open > kMaxScaledGap || -gap_extend > kMaxScaledGap) return false;
    if (m > kColBase || n > kColBase) return false;
    const int64_t bound = (int64_t)(smax > 0 ? smax : 0) * (n < m ? n : m);
    return bound <= kMaxScaledScore;
}

// Device status bits.
constexpr int32_t kStatusReverseMismatch = 1;  // reverse pass lost the score
constexpr int32_t kStatusBadOffsets = 2;       // device offsets decreasing, negative or too long
constexpr int32_t kStatusGuard = 4;            // a guard word around a device buffer changed

// Guard regions (test aid): kGuardBytes of kGuardWord before and after a
// device buffer; a check kernel after the alignment kernels sets
// kStatusGuard when any word of them changed (no trap, no assert).
constexpr uint32_t kGuardWord = 0xA5A5A5A5u;
constexpr size_t kGuardBytes = 4096;
constexpr int kMaxGuards = 32;
struct GuardList {
    uint32_t *ptr[kMaxGuards];
    int32_t words[kMaxGuards];
    int32_t n;
};
cudaError_t launch_guard_fill(const GuardList &g, cudaStream_t s);
cudaError_t launch_guard_check(const GuardList &g, int32_t *status, cudaStream_t s);

// Host planning of the persistent kernel (plan.cpp): which lane-group width
// each pair gets and how many warps start on each width class.
struct PlanPair {
    int32_t id, n, m;
};
struct PlannedClass {
    int log2g;
    std::vector<int32_t> pairs;  // pair ids, largest estimated cost first
    int warps;                   // warps that start on this class
};
std::vector<PlannedClass> plan_classes(const std::vector<PlanPair> &pairs, int n_warps,
                                       int narrow_log2g_hint, double cap_fraction_hint,
                                       int sample_cap = 8192, bool half_tails = false,
                                       int rows = kRows, double strip_overhead = 0.0);
int64_t sweep_steps(int n, int m, int G, int rows = kRows);

// Arithmetic and profile element width of the group kernel: scaled int32
// with an int32 or int8 profile, or two 16-bit cells per 32-bit word.
// The packed form comes with a profile of 32-bit words (scores scaled by 8)
// or, for larger alphabets, of bytes (scaled by 4).
// kPacked16R32: the packed form with 32-bit profile words and 32 rows per
// lane (16 words, two end-key chains), two blocks per SM.
enum class ProfileKind : int {
    kInt32 = 0,
    kInt8 = 1,
    kPacked16 = 2,
    kPacked16Bytes = 3,
    kPacked16R32 = 4
};
constexpr int kNumProfileKinds = 5;
inline bool is_packed(ProfileKind k) {
    return k == ProfileKind::kPacked16 || k == ProfileKind::kPacked16Bytes ||
           k == ProfileKind::kPacked16R32;
}

// Rows per lane of the packed forms with 32-bit profile words (16: 8 words;
// the R32 kind: 32, 16 words).
constexpr int kRowsPacked = 16;
inline int rows_of(ProfileKind k) {
    return k == ProfileKind::kPacked16 ? kRowsPacked : k == ProfileKind::kPacked16R32 ? 32 : kRows;
}

// Whether a pair fits the packed 16-bit form with scores scaled by `scale`
// (8 or 4): every value scale x (score terms) stays in a signed 16-bit
// half and profile scores s - go are non-negative (with a byte profile,
// scale 4, also at most 31, so that 4 (s - go) fits a byte below 128).
inline bool packed_eligible(int n, int m, int smax, int smin, int gap_open, int gap_extend,
                            int scale = 8) {
    if (smin < gap_open || scale * (int64_t)(-gap_extend) > 16384) return false;
    if (scale == 4 && (int64_t)smax - gap_open > 31) return false;
    const int64_t bound = (int64_t)(smax > 0 ? smax : 0) * (n < m ? n : m) +
                          (smax > 0 ? smax : 0) - gap_open;
    return scale * bound <= 32767;
}

// A batch planned on the host (host_plan.cpp): the device tables to upload
// and the launch shapes.
struct HostPlan {
    ProfileKind kind = ProfileKind::kInt32;
    std::vector<PairInfo> pairs;     // persistent kernel, schedule order
    std::vector<ClassInfo> classes;  // its queues
    std::vector<PairInfo> plain;     // one-block-per-pair kernel
    int grid = 0, n_warps = 0;
    int64_t scratch_words = 0;       // strip-boundary words the pairs need
    int32_t slot_words = 0;          // per lane of a group slot (0: per-pair scratch)
    int plain_threads = 32, plain_kmax = 1;
    int64_t q_bytes = 0, r_bytes = 0;  // residues the offsets span
    bool linear = false;     // gap_open == gap_extend: the kernel without E and F
    bool ends_only = false;  // no reverse pass (set by the caller after planning)
};
// Where a HostPlan's tables live on the device.
struct DeviceTables {
    const PairInfo *pairs = nullptr;
    const ClassInfo *classes = nullptr;
    const PairInfo *plain = nullptr;
    int32_t *counters = nullptr;  // kMaxClasses words, zeroed by enqueue_plan
    uint32_t *scratch = nullptr;  // scratch_words words
    int32_t *status = nullptr;
};

// Launchers (return cudaError_t of the launch).
// linear: gap_open == gap_extend, the instantiation without E and F
cudaError_t launch_group(const GroupParams &p, ProfileKind kind, bool linear, int grid,
                         cudaStream_t s);
int group_blocks_per_sm(ProfileKind kind, bool linear, int alphabet, int *smem_bytes);
size_t group_smem_bytes(ProfileKind kind, int alphabet);

cudaError_t launch_plain(const PlainParams &p, int threads, int rows_per_thread_max,
                         cudaStream_t s);
// The plain kernel over a device range (p.range set) with a fixed grid.
cudaError_t launch_plain_range(const PlainParams &p, int threads, int rows_per_thread_max,
                               int grid, cudaStream_t s);
size_t plain_smem_bytes(int threads, int alphabet);

int set_error(int code, const char *msg);  // message for sw_last_error()
// Expands n_res 2-bit packed residues into one byte each (out 4-byte aligned).
cudaError_t enqueue_unpack_2bit(const uint8_t *packed, int64_t n_res, uint8_t *out, int sms,
                                cudaStream_t s);
int ctx_device(const ::sw_ctx *ctx);          // the CUDA device a context works on
// Stream-ordered device memory from the context's workspace pool (release
// with cudaFreeAsync on the same stream).  Returns an sw_status.
int ctx_alloc_async(::sw_ctx *ctx, size_t bytes, cudaStream_t s, void **out);
// Host-to-device upload on s through the context's page-locked staging
// buffer (the host data may be reused when the call returns).
int ctx_upload_async(::sw_ctx *ctx, void *dst, const void *src, size_t bytes, cudaStream_t s);
// The same staging buffer for a caller that writes the upload in place:
// ctx_pinned_acquire waits for the previous upload through it, grows it to
// `bytes` and returns it held; ctx_pinned_commit enqueues the copy of its
// first `bytes` to dst on s and releases it; ctx_pinned_release releases it
// without a copy.  Every acquire is followed by exactly one of the two.
int ctx_pinned_acquire(::sw_ctx *ctx, size_t bytes, void **host);
int ctx_pinned_commit(::sw_ctx *ctx, void *dst, size_t bytes, cudaStream_t s);
void ctx_pinned_release(::sw_ctx *ctx);

// Checks the arguments and plans a batch (no device allocation; queries the
// group kernel's occupancy on the current device).  Returns an sw_status;
// on failure *msg says why.
// Argument and length checks shared by every entry point.  On success
// fills the sequence byte counts and an upper bound on the strip-boundary
// scratch any plan of the batch needs (every group-path pair at the
// narrowest lane-group width).
int check_batch(const int64_t *q_offsets, const int64_t *r_offsets, int32_t n_pairs,
                const int8_t *mat, int32_t A, int32_t go, int32_t ge, int64_t *q_bytes,
                int64_t *r_bytes, int64_t *max_scratch_words, std::string *msg);
// min_pairs_per_warp: the grid of the persistent kernel gets at most one
// warp per this many group-path pairs (1 = lowest latency; 32 >> kMinLog2G
// fills every group of the narrowest width, for a GPU shared with other
// launches).  sample_cap: pairs the planner's schedule simulation looks at
// (fewer plan faster, more plan better).  allow_packed = false keeps the
// scaled int32 arithmetic even where the packed 16-bit form's bound holds.
// blocks_per_sm: occupancy of the group kernel per (profile kind, linear
// gaps, alphabet) (default: the CUDA occupancy query on the current device;
// the host-only plan preview passes an estimate from shared memory).
using BlocksPerSmFn = int (*)(ProfileKind, bool, int, int *);
// group_slots: strip-boundary words in one slot per lane group, sized for
// the batch's largest need (HostPlan::slot_words), instead of per pair.
// rows32: where the packed form with 32-bit profile words applies, take its
// 32-rows-per-lane kernel.
int make_host_plan(const int64_t *q_offsets, const int64_t *r_offsets, int32_t n_pairs,
                   const int8_t *mat, int32_t A, int32_t go, int32_t ge, int32_t mode,
                   int sm_count, int narrow_log2g, double cap_fraction, HostPlan *out,
                   std::string *msg, int min_pairs_per_warp = 1, int sample_cap = 8192,
                   bool allow_packed = true, BlocksPerSmFn blocks_per_sm = group_blocks_per_sm,
                   bool group_slots = false, bool rows32 = false, int blocks_cap = 0);
// Enqueues the kernels of a planned batch on s (queue-head reset included).
cudaError_t enqueue_plan(const HostPlan &hp, const DeviceTables &t, const uint8_t *q,
                         const uint8_t *r, const Outputs &o, const int8_t *mat, int A, int go,
                         int ge, cudaStream_t s);

cudaError_t launch_check_residues(const uint8_t *seqs, int64_t n, int alphabet,
                                  unsigned long long *bad, cudaStream_t s);

}  // namespace swgb
