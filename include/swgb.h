/*
 * swgb: batched Smith-Waterman local alignment with affine (Gotoh) gaps on
 * NVIDIA GB300 (sm_103a).
 *
 * For every (query, reference) pair of a batch the library computes the best
 * local alignment score, its end coordinates (forward pass) and its start
 * coordinates (reverse pass), as ADEPT does with its forward and reverse
 * kernels (paper Section II-B, Fig. 2; Section III-B).
 *
 * Scoring.  Query a_1..a_n indexes matrix rows, reference b_1..b_m columns.
 *   E[i][j] = max(H[i][j-1] + gap_open, E[i][j-1] + gap_extend)
 *   F[i][j] = max(H[i-1][j] + gap_open, F[i-1][j] + gap_extend)
 *   H[i][j] = max(0, H[i-1][j-1] + s(a_i, b_j), E[i][j], F[i][j])
 * with H = 0 and E = F = -infinity on the boundary (Section II-B.1; the
 * affine E update of Fig. 8).  A gap of length k costs
 * gap_open + (k-1) * gap_extend; both are given as signed values <= 0 and
 * must satisfy gap_open <= gap_extend <= 0.
 *
 * Outputs, one int32 each per pair, 0-based inclusive residue indices:
 *   score   S = max H
 *   qend, rend     among cells with H = S: smallest rend, then smallest qend
 *   qstart, rstart among score-S alignments ending at (qend, rend): largest
 *                  rstart, then largest qstart (the reverse pass over the
 *                  reversed prefixes, with the same end rule)
 *   S = 0 (also n = 0 or m = 0): score 0 and all four coordinates -1.
 * The computation is exact integer arithmetic; results are bit-identical to
 * the definition above.
 *
 * Memory.  Sequences are packed residue codes (uint8, each < alphabet_size)
 * concatenated in CSR form: pair p's query is q_seqs[q_offsets[p] ..
 * q_offsets[p+1]) and likewise for the reference.  Unless a function says
 * otherwise, sequence and output pointers are DEVICE pointers owned by the
 * caller; offsets and the scoring matrix are HOST pointers.  The library
 * owns only the context's and plans' device workspaces.
 *
 * Limits.  Each sequence at most SW_MAX_LEN residues; alphabet_size in
 * [1, SW_MAX_ALPHABET]; |gap_open|, |gap_extend| <= SW_MAX_GAP.
 *
 * Errors.  Every entry point returns an sw_status.  Argument errors are
 * detected on the host before anything is enqueued; CUDA failures map to
 * SW_ECUDA.  sw_last_error() returns a message for the calling thread's most
 * recent failure.  No exception crosses this interface.
 *
 * Streams.  `stream` is a cudaStream_t passed as void*; NULL is the legacy
 * default stream.  Work is enqueued asynchronously unless stated otherwise.
 */
#ifndef SWGB_H
#define SWGB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SW_MAX_LEN 65535
#define SW_MAX_ALPHABET 32
#define SW_MAX_GAP 1000000

typedef enum {
    SW_OK = 0,
    SW_EINVAL = -1,   /* bad argument (null pointer, sign, alphabet size) */
    SW_ERANGE = -2,   /* a length, residue or score outside the limits    */
    SW_ENOMEM = -3,   /* device or host allocation failed                 */
    SW_ECUDA = -4,    /* a CUDA runtime call failed                       */
    SW_ETIMEOUT = -5, /* a bounded wait ran out                           */
    SW_EBUDGET = -6   /* a request exceeds the serving memory budget      */
} sw_status;

typedef enum {
    SW_MODE_AUTO = 0,    /* = SW_MODE_BATCHED                               */
    SW_MODE_PLAIN = 1,   /* one thread block per pair, one launch           */
    SW_MODE_BATCHED = 2  /* persistent length-bucketed kernel (+ plain for  */
                         /* pairs beyond its score bound)                   */
} sw_mode;

/* Plan flags. */
#define SW_PLAN_GRAPH 1u /* capture the launch sequence in a CUDA graph and */
                         /* replay it while pointers and stream repeat       */
/* Ends only: score, qend and rend, without the reverse pass (the forward
 * sweep alone, as ADEPT's first kernel, Section III-B).  out_qstart and
 * out_rstart are not written and may be NULL; sw_plan_execute_host copies
 * back only the first 3 x n_pairs values.  Score-only callers use this
 * mode too: the end cell comes with the score at no extra cost. */
#define SW_PLAN_ENDS_ONLY 2u
/* Packed input: q_seqs and r_seqs given to sw_plan_execute /
 * sw_plan_execute_host are 2-bit packed streams (residue k of the stream in
 * byte k >> 2, bits 2 (k & 3) and up; offsets still count residues); needs
 * alphabet_size <= 4.  The plan expands them on the device before the
 * alignment kernels (two small launches inside the same graph); the
 * host-buffer call moves a quarter of the input bytes. */
#define SW_PLAN_PACKED_2BIT 4u
/* Keep the batched kernel on scaled int32 arithmetic.  Without this flag
 * the plan runs the batched kernel in packed 16-bit form (two DP cells per
 * 32-bit word, every value scaled by k) when every pair of the batched path
 * satisfies k x (smax x min(n, m) + smax - gap_open) <= 32767, the smallest
 * matrix entry is >= gap_open and k x |gap_extend| <= 16384, with k = 8
 * (small alphabets, whose profile of 32-bit words leaves two blocks per SM)
 * or k = 4 (a byte profile; also smax - gap_open <= 31); the results are
 * the same either way (sw_plan_arith says which form a plan took). */
#define SW_PLAN_NO_S16X2 8u
/* Strip-boundary scratch per pair instead of per lane group.  A pair whose
 * query or reference spans more than one row strip passes each strip's last
 * row to the next strip through global memory.  By default each lane group
 * of the batched kernel owns one slot of such words, sized for the batch's
 * largest need, and reuses it for every pair it aligns, so the words a
 * launch touches stay few and mostly in L2.  With this flag every such pair
 * gets words of its own (less memory for small batches of long pairs, more
 * DRAM traffic). */
#define SW_PLAN_PAIR_SCRATCH 16u
/* Guard regions (a test aid): every device buffer the plan allocates (pair
 * and class tables, queue heads, strip-boundary scratch, host-call staging)
 * gets 4 KiB of a known pattern before and after it, and each execution
 * enqueues, after the alignment kernels, a check that sets bit 2 of the
 * context's status word (sw_ctx_status) if any guard word changed.  Results
 * are unchanged; nothing traps. */
#define SW_PLAN_GUARDS 32u
/* Where the packed 16-bit form with 32-bit profile words applies (small
 * alphabets), run its kernel with 32 query rows per lane (16 packed words,
 * two blocks per SM) instead of 16 (8 words, three blocks per SM): fewer
 * steps per cell, more padded rows per strip.  Same results. */
#define SW_PLAN_ROWS32 64u

typedef struct sw_ctx sw_ctx;
typedef struct sw_plan sw_plan;

/* Message for the calling thread's most recent failed call ("" if none).
 * The string stays valid until the thread's next failing call. */
const char *sw_last_error(void);

/* Create a context on CUDA device `device` (made current for the call).
 * The context holds device properties, the kernel tuning table and a device
 * status word.  Destroy it after every plan made from it. */
int sw_ctx_create(int32_t device, sw_ctx **out);
int sw_ctx_destroy(sw_ctx *ctx);

/* Number of streaming multiprocessors of the context's device. */
int sw_ctx_sm_count(const sw_ctx *ctx, int32_t *out);

/* *yes = 1 when the context's device reads host memory through the host's
 * page tables over a coherent link (cudaDevAttrPageableMemoryAccessUses-
 * HostPageTables), so sw_plan_execute_host reads page-locked inputs in
 * place; 0 otherwise (or after sw_ctx_set_host_in_place(ctx, 0)). */
int sw_ctx_host_in_place(const sw_ctx *ctx, int32_t *yes);

/* enable = 0: host-buffer executions and one-shot calls on this context
 * copy page-locked host inputs to the device (copy engines) instead of
 * letting the kernels read them over the host link; 1 (the default where
 * the device supports it): read them in place.  Results are the same; the
 * faster transport depends on the link's load (reads in place overlap the
 * transfer with the alignment, copies keep the kernels on device memory).
 * Errors: SW_EINVAL. */
int sw_ctx_set_host_in_place(sw_ctx *ctx, int32_t enable);

/* Synchronise the context's device, return its device status word in
 * *status (0 = no inconsistency detected by any kernel; bit 0 = a reverse
 * pass did not reproduce its forward score; bit 1 = a one-shot call met
 * device offsets that were negative, decreasing or more than SW_MAX_LEN
 * apart, and gave those pairs the "no alignment" outputs; bit 2 = a guard
 * word of a plan made with SW_PLAN_GUARDS, or of a one-shot workspace with
 * guards on, changed) and clear it. */
int sw_ctx_status(sw_ctx *ctx, int32_t *status);

/* Guard regions around the one-shot calls' workspace parts (tables, sort
 * buffers, strip-boundary slots), checked after each call's kernels as for
 * SW_PLAN_GUARDS (on = 1; 0 = off, the default).  A test aid. */
int sw_ctx_set_guards(sw_ctx *ctx, int32_t on);

/* The context sw_align_batch uses on `device` (created on first use, owned
 * by the library until the process exits: do not destroy it).  Its status
 * word reports on sw_align_batch's work (sw_ctx_status). */
int sw_default_ctx(int32_t device, sw_ctx **out);

/* Batched-path tuning for plans created afterwards.  narrow_log2g = -1
 * (default): the planner chooses the lane-group width of the bulk of the
 * pairs and the long-pair cap itself, by simulating the schedule of a few
 * candidates.  narrow_log2g in [0, 5] fixes the bulk width G = 2^narrow_log2g;
 * pairs whose serial sweep under it exceeds cap_fraction x the mean load of
 * a group go to wider groups (cap_fraction > 0; a huge value keeps one
 * width for all pairs). */
int sw_ctx_set_tuning(sw_ctx *ctx, int32_t narrow_log2g, double cap_fraction);

/* Batched kernel form for plans created afterwards (a plan's flags still
 * override): arith = -1 (default: the packed 16-bit form wherever its bound
 * holds), 0 (scaled int32 always), 1 (packed where legal); rows = 16 or 32
 * rows per lane for the packed form with 32-bit profile words (32 as
 * SW_PLAN_ROWS32); blocks_per_sm = resident blocks per SM of the persistent
 * kernel (0, the default: as many as its registers and shared memory allow;
 * a larger value than fits means the same).  sw_autotune sets all three. */
int sw_ctx_set_form(sw_ctx *ctx, int32_t arith, int32_t rows, int32_t blocks_per_sm);

/* The context's current tuning (any pointer may be NULL). */
int sw_ctx_get_tuning(const sw_ctx *ctx, int32_t *narrow_log2g, double *cap_fraction,
                      int32_t *arith, int32_t *rows, int32_t *blocks_per_sm);

/*
 * Plan a batch.  q_offsets and r_offsets are HOST arrays of n_pairs + 1
 * non-decreasing int64 offsets; score_matrix is a HOST row-major
 * alphabet_size x alphabet_size int8 table (row = query residue).  The plan
 * sorts the pairs by cost (longest first), buckets them into warp tasks,
 * uploads its tables and allocates the device scratch the batch needs.
 * Blocking; nothing is enqueued on any stream.
 * Errors: SW_EINVAL (null pointer, n_pairs < 0, bad gaps/alphabet/mode),
 * SW_ERANGE (a length above SW_MAX_LEN or offsets decreasing), SW_ENOMEM,
 * SW_ECUDA.
 */
int sw_plan_create(sw_ctx *ctx, const int64_t *q_offsets, const int64_t *r_offsets,
                   int32_t n_pairs, const int8_t *score_matrix, int32_t alphabet_size,
                   int32_t gap_open, int32_t gap_extend, int32_t mode, uint32_t flags,
                   sw_plan **out);

/*
 * Run a plan on `stream`.  q_seqs / r_seqs are DEVICE pointers to the
 * residues the plan's offsets index; the five outputs are DEVICE arrays of
 * n_pairs int32, written at each pair's position in the batch.  Residue
 * codes are clamped to alphabet_size - 1 on the device (use
 * sw_check_residues to validate).  The batched kernel reads residues in
 * whole 16-byte aligned chunks, so it may read up to 15 bytes before or
 * after a sequence; both buffers must lie in memory from the CUDA
 * allocators (whose allocations cover whole aligned 16-byte chunks), which
 * every device pointer of a cudaMalloc'd or PyTorch tensor does.
 * Asynchronous; the plan may be executed
 * again once this execution has been ordered before the next on the same
 * stream.  Executions of one plan on different streams must not overlap.
 */
int sw_plan_execute(sw_plan *plan, const uint8_t *q_seqs, const uint8_t *r_seqs,
                    int32_t *out_score, int32_t *out_qend, int32_t *out_rend,
                    int32_t *out_qstart, int32_t *out_rstart, void *stream);

/*
 * Run a plan on HOST buffers: copies q_seqs[0 .. q_offsets[n_pairs]) and
 * r_seqs[0 .. r_offsets[n_pairs]) (offsets as planned) to plan-owned device
 * buffers on `stream`, executes, copies the results to out_host (5 x n_pairs
 * int32: all scores, then all qend, rend, qstart, rstart) and synchronises
 * `stream`.  Page-locked host memory makes the copies asynchronous DMA.
 * The staging buffers are allocated on the first call and kept by the plan.
 * When the context's device reads host memory over a coherent link
 * (sw_ctx_host_in_place says 1: NVLink-C2C on Grace) and both sequence
 * buffers are page-locked (cudaHostAlloc / cudaHostRegister), the kernels
 * read them in place instead: each residue crosses the link once, while the
 * alignment runs, and no input copy precedes the kernels.
 */
int sw_plan_execute_host(sw_plan *plan, const uint8_t *q_seqs, const uint8_t *r_seqs,
                         int32_t *out_host, void *stream);

/* Shape of a plan (any pointer may be NULL): n_group_pairs pairs on the
 * persistent kernel, n_plain pairs on the one-block-per-pair kernel,
 * launches = kernels one execution enqueues, scratch_bytes = device scratch
 * for strip boundaries. */
int sw_plan_info(const sw_plan *plan, int32_t *n_group_pairs, int32_t *n_plain,
                 int32_t *launches, int64_t *scratch_bytes);

/* Arithmetic of a plan's batched kernel: *arith = SW_ARITH_S32 (scaled
 * int32, one cell per instruction) or SW_ARITH_S16X2 (packed 16-bit, two
 * cells per instruction).  Plans without batched-path pairs report
 * SW_ARITH_S32. */
#define SW_ARITH_S32 0
#define SW_ARITH_S16X2 1
int sw_plan_arith(const sw_plan *plan, int32_t *arith);
/* Query rows per lane of a plan's batched kernel (16 or 32). */
int sw_plan_rows(const sw_plan *plan, int32_t *rows);

/* Test aid for plans made with SW_PLAN_GUARDS: overwrite one word in the
 * middle of guard region `region` (0 .. 2 x the plan's guarded buffers - 1)
 * with a value other than the guard pattern (a host-side copy into the
 * plan's own allocation, after synchronising the device), so that the next
 * execution's check must report it.  SW_EINVAL if the plan has no such
 * region. */
int sw_plan_poison_guard(sw_plan *plan, int32_t region);

int sw_plan_destroy(sw_plan *plan);

/*
 * Host-only preview of how sw_plan_create would plan a batch (no CUDA call,
 * no allocation; for inspection and tests on machines without a GPU).
 * Arguments as sw_plan_create (offsets and matrix on the HOST), plus the SM
 * count of the device to plan for and the tuning (as sw_ctx_set_tuning);
 * the group kernel's occupancy is estimated from its shared memory (228 KB
 * per SM, 1 KB reserved per block) and its register bound (3 blocks).
 * Outputs: *out_kind = the batched kernel's form: 0 = int32 with an int32
 * profile, 1 = int32 with an int8 profile, 2 = packed 16-bit with a profile
 * of 32-bit words, 3 = packed 16-bit with a byte profile; pair_log2g[i] =
 * log2 of the lane-group width pair i is aligned with, or -1 for the
 * one-block-per-pair kernel; pair_rank[i] = its position in that kernel's
 * queue (group pairs: in its width class, longest first).
 * Errors: as sw_plan_create; SW_EINVAL for bad tuning or NULL outputs.
 */
int sw_plan_preview(const int64_t *q_offsets, const int64_t *r_offsets, int32_t n_pairs,
                    const int8_t *score_matrix, int32_t alphabet_size, int32_t gap_open,
                    int32_t gap_extend, int32_t mode, uint32_t flags, int32_t sm_count,
                    int32_t narrow_log2g, double cap_fraction, int32_t *out_kind,
                    int32_t *pair_log2g, int32_t *pair_rank);

/*
 * Measured tuning of the batched path for a batch (blocking).  Runs the
 * batch - offsets and score_matrix on the HOST as for sw_plan_create,
 * q_seqs/r_seqs on the DEVICE, `out` a DEVICE scratch array of 5 x n_pairs
 * int32 that receives the results - once per candidate tuning (bulk
 * lane-group width 2, 4, 8, 16 or 32 with long-pair caps 0.25, 0.5, 1 or none, and
 * the planner's own choice; for a batch that takes the packed form with
 * 32-bit profile words, each of those also with 32 rows per lane and in the
 * scaled int32 form), then the fastest with two resident blocks per SM
 * instead of three, keeps the fastest and sets it on ctx with
 * sw_ctx_set_tuning and sw_ctx_set_form (sw_ctx_get_tuning reads it back).
 * With a non-NULL cache_path the choice is looked up first and stored after
 * measuring in that JSON file, keyed by GPU name, SM
 * count and a signature of the batch (pair count, length sums, maxima and
 * histograms, scoring); a hit skips the measurement.  Outputs (may be
 * NULL): the chosen narrow_log2g and cap_fraction and its time in ms.
 */
int sw_autotune(sw_ctx *ctx, const int64_t *q_offsets, const int64_t *r_offsets,
                int32_t n_pairs, const int8_t *score_matrix, int32_t alphabet_size,
                int32_t gap_open, int32_t gap_extend, const uint8_t *q_seqs,
                const uint8_t *r_seqs, int32_t *out, const char *cache_path, void *stream,
                int32_t *chosen_log2g, double *chosen_frac, double *chosen_ms);

/* sw_autotune for plans that will be made with plan `flags`: the candidates
 * are planned with its SW_PLAN_ENDS_ONLY and SW_PLAN_NO_S16X2 bits (the
 * other bits are ignored; q_seqs/r_seqs are one byte per residue), and the
 * cache key includes those bits.  sw_autotune = flags 0. */
int sw_autotune_ex(sw_ctx *ctx, const int64_t *q_offsets, const int64_t *r_offsets,
                   int32_t n_pairs, const int8_t *score_matrix, int32_t alphabet_size,
                   int32_t gap_open, int32_t gap_extend, const uint8_t *q_seqs,
                   const uint8_t *r_seqs, int32_t *out, uint32_t flags, const char *cache_path,
                   void *stream, int32_t *chosen_log2g, double *chosen_frac, double *chosen_ms);

/*
 * One-shot alignment of a batch whose sequences AND offsets are on the
 * DEVICE (score_matrix on the HOST): the forward and reverse passes of
 * every pair, as ADEPT's batch call (Section III-B), planned on the device.
 * Where the device reads host memory coherently (sw_ctx_host_in_place: a
 * GB300's host link), the sequences and offsets may instead be page-locked
 * host buffers (cudaMallocHost / cudaHostRegister), read in place by the
 * kernels; the outputs stay device memory.
 *
 * Asynchronous: the call checks its arguments, enqueues everything on
 * `stream` and returns SW_OK without waiting for the device or reading
 * anything back.  The kernels it enqueues read the offsets, give every pair
 * its route and lane-group width (the same rules and cost model as
 * sw_plan_create's planner, with the bulk width and cap of the context's
 * tuning, else 8 lanes and half the mean load, instead of its simulated
 * candidate search), sort the pairs longest first per width with a radix
 * sort, build the queue tables and run the alignment kernels.  Device
 * offsets that are negative, decreasing or more than SW_MAX_LEN apart give
 * the pair the "no alignment" outputs and set bit 1 of the context's status
 * word (sw_ctx_status; for sw_align_batch, the context sw_default_ctx
 * returns).
 *
 * Workspace: tables and sort buffers of about 52 bytes per pair plus the
 * strip-boundary slots of the lane groups (1028 words per lane, about 240 MB
 * on a GB300), taken stream-ordered from a memory pool of the context that
 * keeps freed memory for later calls; a pair whose longer sequence has
 * more than about 16,400 residues (beyond the widest group's slot) takes
 * the plain kernel.  Calls on different streams may overlap.  For repeated batches of
 * one shape, sw_plan_create + sw_plan_execute plan once on the host.
 * Errors (host-side, before anything is enqueued): SW_EINVAL for NULL
 * pointers, n_pairs < 0, a bad alphabet size, gaps or mode; SW_ENOMEM when
 * the workspace cannot be had; SW_ECUDA.
 */
int sw_align_batch(const uint8_t *q_seqs, const int64_t *q_offsets,
                   const uint8_t *r_seqs, const int64_t *r_offsets, int32_t n_pairs,
                   const int8_t *score_matrix, int32_t alphabet_size,
                   int32_t gap_open, int32_t gap_extend,
                   int32_t *out_score, int32_t *out_qend, int32_t *out_rend,
                   int32_t *out_qstart, int32_t *out_rstart, void *stream);

/*
 * As sw_align_batch with an explicit context (its tuning, status word and
 * workspace pool) and mode (sw_mode; SW_MODE_PLAIN sends every pair to the
 * one-block-per-pair kernel).
 */
int sw_align_batch_ex(sw_ctx *ctx, const uint8_t *q_seqs, const int64_t *q_offsets,
                      const uint8_t *r_seqs, const int64_t *r_offsets, int32_t n_pairs,
                      const int8_t *score_matrix, int32_t alphabet_size,
                      int32_t gap_open, int32_t gap_extend, int32_t mode,
                      int32_t *out_score, int32_t *out_qend, int32_t *out_rend,
                      int32_t *out_qstart, int32_t *out_rstart, void *stream);

/*
 * Validate residue codes on the device: counts the codes >= alphabet_size in
 * seqs[0 .. n) into *bad_count (a DEVICE int64, overwritten).  Asynchronous.
 */
int sw_check_residues(const uint8_t *seqs, int64_t n, int32_t alphabet_size,
                      int64_t *bad_count, void *stream);

/*
 * Allocation-free batched alignment.  The paper has no counterpart: this is
 * for callers that cannot allocate device memory when they align - code
 * running where another component (a framework's caching allocator, a
 * fixed-size arena) already owns the device's memory budget, or a
 * latency-critical loop that must not stall on the implicit device
 * synchronisation of cudaMalloc/cudaFree.
 *
 * Same computation, outputs and kernels as sw_plan_create +
 * sw_plan_execute in SW_MODE_AUTO, but the call allocates no device memory:
 * its tables, queue heads and strip-boundary scratch live in one fixed
 * module array of about 37 MiB that every GPU that loads the library keeps
 * until the process exits.  q_seqs, r_seqs and the five outputs are DEVICE
 * pointers owned by the caller; q_offsets, r_offsets and score_matrix are
 * HOST arrays, as for sw_plan_create.
 *
 * Limits: at most SW_STATIC_MAX_PAIRS pairs per call, and the pairs whose
 * query or reference spans more than one row strip (the reverse sweep takes
 * the reference as rows) need about 2 x (longer sequence length) boundary
 * words each, at most SW_STATIC_MAX_BOUNDARY_WORDS in total; a batch beyond
 * either is rejected with SW_ERANGE before anything is enqueued (split it).
 *
 * The first call on a device resolves the array's device address on that
 * device and keeps it for the life of the process; after cudaDeviceReset
 * (or from another CUDA context on that device) the kept address is no
 * longer valid, so use this entry point only from the context that made the
 * first call.  Every call uses the same array (it keeps the previous call's
 * contents and clears what must start at zero), so calls whose GPU work
 * overlaps - on different streams or threads - race with each other: order
 * them, e.g. on one stream.  The work is enqueued on `stream` and the call
 * returns; the host arrays may be reused once it has returned.  The call
 * copies its pair tables from host memory it frees on return, so it cannot
 * be captured into a CUDA graph: on a capturing stream it returns SW_EINVAL.
 */
#define SW_STATIC_MAX_PAIRS 65536
#define SW_STATIC_MAX_BOUNDARY_WORDS (8 << 20)
int sw_align_batch_static(const uint8_t *q_seqs, const int64_t *q_offsets,
                          const uint8_t *r_seqs, const int64_t *r_offsets, int32_t n_pairs,
                          const int8_t *score_matrix, int32_t alphabet_size,
                          int32_t gap_open, int32_t gap_extend,
                          int32_t *out_score, int32_t *out_qend, int32_t *out_rend,
                          int32_t *out_qstart, int32_t *out_rstart, void *stream);

/* Status word of sw_align_batch_static's kernels (bit 0 = a reverse pass
 * did not reproduce its forward score; 0 = no inconsistency), collected
 * over every call since it was last read: waits for `stream`, copies the
 * word from the fixed module array into *status (a HOST word) and clears it
 * on `stream`.  Allocates nothing.  Call it on the stream of the calls it
 * reports on. */
int sw_static_status(int32_t *status, void *stream);

/*
 * Serving: continuous batching of alignment requests (one device, blocking
 * calls are bounded by timeouts).
 *
 * sw_server_create: a server on ctx's device with a device-memory budget of
 * budget_bytes (allocated once, at creation, as the arena that holds the
 * resident pools and every launch's sequences, offsets, planning workspace
 * and outputs), at most `streams` launches on the GPU at a time (one stream
 * each, 1..64), and a pinned host staging pool of staging_bytes.  A worker
 * thread forms launches whenever a stream slot is free: the oldest queued
 * request plus the later queued requests from the same source (the same
 * resident pool, or staged sequences with the same matrix and gap costs),
 * up to 262144 pairs and 4e9 cells per launch and what the arena has left.
 * Each launch is planned on the device, as sw_align_batch plans (no host
 * planning); launches on different slots overlap on the device.
 *
 * sw_server_submit: queue a request given as HOST arrays (sequences,
 * offsets, matrix; copied into the staging pool before the call returns, so
 * the caller may reuse them).  Waits up to timeout_ms for staging space.
 * Errors: SW_EINVAL/SW_ERANGE as sw_plan_create; SW_EBUDGET if the request
 * alone needs more than the budget (less the pools) or the staging pool;
 * SW_ETIMEOUT.
 *
 * sw_server_add_pool: upload a batch (HOST arrays, as sw_server_submit) into
 * the budget once, as resident pool *pool_id, for the server's lifetime
 * (blocking copy).  SW_EBUDGET if it does not fit the free budget.
 * sw_server_submit_pool: queue a request for pairs [first_pair, first_pair +
 * n_pairs) of a resident pool, aligned with the pool's scoring; only the
 * pairs' offsets go up and the results come back.  SW_ERANGE for a range
 * outside the pool; otherwise as sw_server_submit.
 *
 * sw_server_wait: wait up to timeout_ms for a request, copy its results to
 * out_host (5 x n_pairs int32: scores, qend, rend, qstart, rstart) and
 * forget it.  SW_ETIMEOUT leaves it pending (wait again later).  If done_ns
 * is not NULL it receives the CLOCK_MONOTONIC time, in nanoseconds, at
 * which the worker saw the request's work finish on the GPU (results back
 * in the staging pool), so that a client can measure latency from its own
 * arrival times on the same clock.
 *
 * Results equal those of sw_plan_execute on the same batch.  The paper runs
 * fixed batches only (Section 3); the server is this library's addition for
 * callers whose pairs arrive over time.
 */
typedef struct sw_server sw_server;
int sw_server_create(sw_ctx *ctx, int64_t budget_bytes, int32_t streams, int64_t staging_bytes,
                     sw_server **out);
int sw_server_submit(sw_server *server, const uint8_t *q_seqs, const int64_t *q_offsets,
                     const uint8_t *r_seqs, const int64_t *r_offsets, int32_t n_pairs,
                     const int8_t *score_matrix, int32_t alphabet_size, int32_t gap_open,
                     int32_t gap_extend, int32_t timeout_ms, int64_t *request_id);
int sw_server_add_pool(sw_server *server, const uint8_t *q_seqs, const int64_t *q_offsets,
                       const uint8_t *r_seqs, const int64_t *r_offsets, int32_t n_pairs,
                       const int8_t *score_matrix, int32_t alphabet_size, int32_t gap_open,
                       int32_t gap_extend, int32_t *pool_id);
int sw_server_submit_pool(sw_server *server, int32_t pool_id, int64_t first_pair,
                          int32_t n_pairs, int32_t timeout_ms, int64_t *request_id);
int sw_server_poll(sw_server *server, int64_t request_id, int32_t *done);
int sw_server_wait(sw_server *server, int64_t request_id, int32_t timeout_ms, int32_t *out_host,
                   int64_t *done_ns);
int sw_server_stats(sw_server *server, int64_t *completed, int64_t *in_flight, int64_t *queued,
                    int64_t *device_bytes_in_use, int64_t *device_bytes_peak);
/* Launches the worker has started so far, the pairs they held and the host
 * milliseconds spent preparing them (offsets, copies and enqueueing; the
 * planning itself runs on the device) (any pointer may be NULL). */
int sw_server_launches(sw_server *server, int64_t *launches, int64_t *pairs_launched,
                       double *plan_ms);
int sw_server_destroy(sw_server *server);

/*
 * 2-bit packing of DNA codes (0..3), four per byte, first residue in the low
 * bits.  sw_pack_2bit: HOST arrays, (n_res + 3) / 4 bytes out; SW_ERANGE on a
 * code above 3.  sw_unpack_2bit: DEVICE arrays (codes 4-byte aligned),
 * enqueued on `stream`.
 */
int sw_pack_2bit(const uint8_t *codes, int64_t n_res, uint8_t *packed);
int sw_unpack_2bit(const uint8_t *packed, int64_t n_res, uint8_t *codes, void *stream);

/*
 * Traceback: the alignment itself (Fig. 2(c)'s traceback from the maximal
 * cell), as a CIGAR per pair, for a batch already aligned.
 *
 * results: HOST, 5 x n_pairs int32 rows (score, qend, rend, qstart,
 * rstart), as sw_plan_execute writes them.  For each pair with score > 0
 * the alignment is the best global alignment, under the same affine
 * scoring, of q[qstart..qend] against r[rstart..rend] (its score is the
 * pair's score); among co-optimal ones the walk back from the last cell
 * takes the diagonal first, then a gap in the query (D), then a gap in the
 * reference (I), and inside a gap steps back out where the run opened.
 * Ops are run-length encoded as (length << 4) | code, code M = 0, I = 1
 * (query residue only), D = 2 (reference residue only), first op first.
 *
 * sw_cigar_capacity: HOST helper; offsets[0..n_pairs] with room
 * (qend - qstart + 1) + (rend - rstart + 1) ops for each aligned pair, 0
 * for the others.
 * sw_traceback: q_seqs, r_seqs, out_ops, out_n_ops on the DEVICE; offsets,
 * matrix, results and cigar_offsets on the HOST (read during the call).
 * Pair p's ops go to out_ops[cigar_offsets[p] ..], their count to
 * out_n_ops[p] (0 when the score is 0).  Asynchronous: the work is enqueued
 * on `stream` and the call returns (its host preparation, split over up to
 * 8 worker threads for large batches, is done by then).  Spans of at most
 * 512 query residues whose scores fit int32 with room and whose s - go fit a
 * signed byte take the fast path (a lane group per span, 10 to 16 rows per
 * lane, four choice bits per cell, then the group walks the span back);
 * longer spans the general one.  Scratch (half a byte per cell of the fast
 * path's spans, rounded up to its rows; at most about 1 GiB per launch of
 * the general path's choice bytes) comes from the context's workspace pool,
 * stream-ordered.
 * Errors: SW_EINVAL (bad arguments), SW_ERANGE (offsets negative or
 * decreasing, a length above SW_MAX_LEN, coordinates outside a pair, or room
 * below the pair's need), SW_ENOMEM, SW_ECUDA.
 */
int sw_cigar_capacity(const int32_t *results, int32_t n_pairs, int64_t *offsets);
int sw_traceback(sw_ctx *ctx, const uint8_t *q_seqs, const int64_t *q_offsets,
                 const uint8_t *r_seqs, const int64_t *r_offsets, int32_t n_pairs,
                 const int8_t *score_matrix, int32_t alphabet_size, int32_t gap_open,
                 int32_t gap_extend, const int32_t *results, const int64_t *cigar_offsets,
                 uint32_t *out_ops, int32_t *out_n_ops, void *stream);

/*
 * Traceback of a batch whose results are already on the device (Fig. 2(c),
 * the same alignments, ops and rule as sw_traceback), with the span
 * classification done by kernels instead of host threads.
 *
 * sw_cigar_capacity_device: results (5 x n_pairs int32 rows, as the
 * alignment calls write them) and offsets[0..n_pairs] on the DEVICE; writes
 * the same offsets as sw_cigar_capacity, offsets[n_pairs] the total.
 * Asynchronous on `stream`.  Errors: SW_EINVAL, SW_ECUDA.
 *
 * sw_traceback_device: q_seqs, q_offsets, r_seqs, r_offsets, results,
 * cigar_offsets, out_ops and out_n_ops on the DEVICE; score_matrix on the
 * host.  Three kernels classify the spans (fast or general path, lane-group
 * class, span length), sort the fast-path records by class and length and
 * lay out their choice words; the call then waits for them (and so for the
 * work queued on `stream` before it), reads back a summary of under 1 KB
 * (and the general-path records, when there are any), and enqueues the
 * fill and walk kernels, which run asynchronously.  Scratch as for
 * sw_traceback, from the context's pool, stream-ordered.  Offsets and
 * results are checked on the device: SW_ERANGE names the smallest bad pair
 * (offsets negative or decreasing, a length above SW_MAX_LEN, coordinates
 * outside the pair, or room below its need) and then nothing is enqueued
 * beyond the cleared out_n_ops.  The call cannot be captured in a CUDA
 * graph (it waits on the stream): on a stream being captured it returns
 * SW_EINVAL and enqueues nothing.  Other errors: SW_EINVAL, SW_ENOMEM,
 * SW_ECUDA.
 */
int sw_cigar_capacity_device(const int32_t *results, int32_t n_pairs, int64_t *offsets,
                             void *stream);
int sw_traceback_device(sw_ctx *ctx, const uint8_t *q_seqs, const int64_t *q_offsets,
                        const uint8_t *r_seqs, const int64_t *r_offsets, int32_t n_pairs,
                        const int8_t *score_matrix, int32_t alphabet_size, int32_t gap_open,
                        int32_t gap_extend, const int32_t *results, const int64_t *cigar_offsets,
                        uint32_t *out_ops, int32_t *out_n_ops, void *stream);

/*
 * Integer issue-rate microbenchmark on `device` (made current for the call;
 * synchronous).  op: 0 = 32-bit add, 1 = 32-bit max, 2 = __viaddmax_s32
 * (add then max), 3 = __vimax3_s32_relu, 4 = __viaddmax_s16x2,
 * 5 = __vimax_s32_relu, 6 = __vimax3_s16x2, 7 = __viaddmax_s16x2_relu.  Runs 64 warps per SM, each thread 8 independent
 * chains of `iters` x 16 instructions, and returns whole-device
 * instructions per second (per 32-bit lane) in *ops_per_s and the timed
 * duration in *seconds (may be NULL).  This measures the denominator of the
 * alignment kernels' roofline; the paper has no counterpart.
 */
int sw_microbench_int(int32_t op, int32_t device, int64_t iters, double *ops_per_s,
                      double *seconds);

#ifdef __cplusplus
}
#endif

#endif /* SWGB_H */
