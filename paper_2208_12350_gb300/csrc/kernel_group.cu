// Persistent, length-bucketed batched kernel: the hot path.
//
// Work split.  The plan sorts pairs into classes by lane-group width G (32,
// 16, ..., 2; longest sweeps first) and, inside a class, by cost.  A warp
// takes one class at a time and splits into 32/G groups of G lanes.  Each
// group independently pulls a pair from its class queue, runs the forward
// sweep, then the reverse sweep of the same pair, then pulls the next pair,
// so groups never wait for one another's pairs.
//
// Sweep.  Lane t of a group holds query rows [t*R, t*R + R) of the current
// row strip in registers and walks the reference columns, lane t on column
// j = step - t: the anti-diagonal wavefront of ADEPT (Section II-B.2,
// Fig. 3) with R rows per lane.  The H and F values of the row above arrive
// by one register shuffle per value per step from lane t-1, executed by
// every lane alike, so the exchange never diverges (the lesson of GEVO's
// edits 5, 6, 8 and 10, Section VI-A).  Lane 0 takes them from the strip
// boundary instead: H = 0 / F = -infinity above the first strip (Section
// II-B.1's boundary row), and for later strips the last row of the previous
// strip, which lane G-1 wrote to global scratch.  Queries longer than G*R
// rows take several strips ("passes").  (A build option, SWGB_SPLIT_ROWS,
// runs a lane's two row halves a column apart instead; measured slower.)
//
// Staging.  Reference residues and strip-boundary words move in 16-byte
// pieces (the profile build reads its rows' residues directly).  Each group has
// three small rings in shared memory: reference residues (128 bytes, filled
// by its lane 0 with cp.async a few 4-step blocks ahead; each lane then
// reads its residue with a shared-memory load), the previous strip's
// boundary words (cp.async, same distance), and this strip's boundary words
// (lane G-1 stores one word per step and writes each completed aligned
// group of four to global memory with one 16-byte store).
//
// Every lane runs the same instruction stream on every step: columns outside
// a lane's range, idle groups and rows past the end of the query are
// computed with a pad residue whose scores are very negative, instead of
// being branched around.  Such cells never beat a real cell: their values
// come from real cells at an earlier column (or the same column and a
// smaller row) through non-positive steps, and ties go to the smaller
// column, then the smaller row.  Before a lane's first column the pad
// column leaves H = 0 and E = go, which gives the same first real column as
// the E = -infinity boundary.
//
// Recurrence (Section II-B.1, Fig. 8), per cell, with H kept as H + go
// (call it X) so that both gap updates read it directly:
//   E   = viaddmax(E, ge, X_left)                E = max(E + ge, H_left + go)
//   F   = viaddmax(F_up, ge, X_up)               F = max(F_up + ge, H_up + go)
//   X   = vimax3_relu(X_diag + s', E, F) + go    H = max(H_diag + s, E, F, 0)
//   K   = viaddmax(X, kColBase - j - go, K)      end-cell key of the row
// with s' = s - go from the profile.  Five maxes per cell (E, F, two for
// the three-way max with 0, the key) run on the integer ALU pipe; the adds
// fuse into them or issue on the FMA pipe.  All scores are scaled by 2^16,
// so K = (H << 16) | (kColBase - j) orders cells by larger H, then smaller
// column, at one instruction per cell; rows are compared in ascending order
// with a strict "greater" so the smaller row wins ties.  The plan sends a
// pair here only when smax * min(n, m) <= 32766, |go|, |ge| <= 16383 and
// n, m <= kColBase, which keeps every scaled value and key inside int32 and
// the column part in [0, 65535) also on the pad columns a lane computes
// before its first column (j >= -63).
//
// Packed 16-bit form (PK).  Two cells per instruction: word k of a lane
// holds row k in its low half (at column j) and row R/2 + k in its high half
// (one column behind, j - 1), the split-row schedule with both halves in one
// register, so every packed max serves two independent row chains.  Scores
// are scaled by 8 and held as non-negative 16-bit values:
//   Hs = 8 H,   Es = 8 (E - go),   Fs = 8 (F - go),   s' = 8 (s - go) >= 0
//   Es  = viaddmax2(Es, 8 ge, Hs_left)              E - go = max(E - go + ge, H_left)
//   Fs  = viaddmax2(Fs_up, 8 ge, Hs_up)             F - go = max(F_up - go + ge, H_up)
//   Hs  = viaddmax2_relu(vimax3_2(Hs_diag + s', Es, Fs), 8 go, 0)
//                                                   H = max(H_diag + s, E, F, 0)
// Hs_diag + s' is a plain 32-bit add: both halves are non-negative and their
// sums stay below 2^15, so no carry crosses from the low half to the high
// one; s' comes from two profile words (low-half rows against column j's
// residue, high-half rows against column j - 1's) whose other halves are 0.
// The end cell: the low 3 bits of every Hs are 0, so Hs_k + (7 - k) is a
// carry-free 32-bit add and a chain acc = vimax3_2(Hs_k + 7 - k,
// Hs_k+1 + 6 - k, acc) over a lane's 8 words (one three-way max per pair of
// words) gives, per half, the column's largest score with the smallest row
// holding it (row code 7 - k).  The chain starts from a threshold T = (8 best + 7): acc differs
// from T in a half exactly when that half's best score grew at this column,
// and the (column, acc) pair of that step is recorded, so each half ends
// with its largest score, the first column reaching it and the smallest row
// there.  The transposed reverse sweep starts T at 8 S - 1 and keeps it at
// acc: a half records the smallest row holding S and that row's first
// column.  Rows past n and columns outside [0, m) take s' = 0 (s = go): such
// a cell's value is reached through non-positive steps from a real cell
// with a smaller (column, row) pair, so its record never wins.  The plan
// takes this form only when 8 (smax min(n, m) + smax - go) <= 32767,
// smin >= go and 8 |ge| <= 16384, which keeps every value in 16 bits.
// Large alphabets (protein) use a byte profile instead (P8 with PK): s' =
// 4 (s - go) < 128 per byte, scores scaled by 4, 2-bit row codes in chains
// of 4 words, and one sign-replicating byte permute per word that moves the
// two rows' bytes into the halves (bound 4 (smax min(n, m) + smax - go) <=
// 32767, smax - go <= 31).
//
// Reverse pass (Fig. 2(c)): the same sweep over the reversed prefixes
// a_qend..a_0 and b_rend..b_0, transposed: the reversed reference prefix
// gives the rows (in registers, strip by strip) and the reversed query
// prefix the columns, with the substitution matrix read transposed.  The
// start rule wants, among the cells of score S, the largest rstart (the
// smallest reversed reference index, here a row) and then the largest
// qstart (the smallest column).  Strips run in row order, so the sweep ends
// with the first strip that holds a cell of score S: its smallest such row,
// and that row's smallest such column, which the per-row end key already
// gives.  The rows below that strip are never computed; had the reverse
// sweep kept the query as rows, every strip before the one holding the
// start would have run over all rend + 1 columns.
#include <algorithm>
#include <mutex>
#include <type_traits>

#include "sw_internal.h"

namespace swgb {
namespace {

constexpr unsigned kFull = 0xffffffffu;
// Steps per block (one staging round, one strip-end check): 8 for the
// packed form (12 % faster than 4 on 100k and 200k DNA pairs: fewer
// per-block instructions per cell) and the int8-profile int32 form (+2 % on
// 20k protein pairs), 4 for the int32-profile int32 form (at 8 it spills).
#ifndef SWGB_GROUP_UNROLL
#define SWGB_GROUP_UNROLL 4
#endif
#ifndef SWGB_PACKED_UNROLL
#define SWGB_PACKED_UNROLL 8
#endif
template <bool P8, bool PK>
__host__ __device__ constexpr int unroll_of() {
    return (PK || P8) ? SWGB_PACKED_UNROLL : SWGB_GROUP_UNROLL;
}
#ifndef SWGB_STEP_ORDER_FENCE
#define SWGB_STEP_ORDER_FENCE 1
#endif
#ifndef SWGB_SPLIT_ROWS
#define SWGB_SPLIT_ROWS 0
#endif
// Packed form, end-key chain of a column: 0 = one viaddmax per word
// (acc = max(h_k + code_k, acc)); 1 = words in pairs, the sums h_k + code_k
// as plain adds and one three-way max per pair (half the ALU-pipe maxes);
// 2 = as 1 with the adds forced onto the FMA pipe (multiply-add by a one
// the compiler cannot see).  Measured with the same tuning on one GB300:
// 1 is 1.9 % faster than 0 on 100k DNA pairs and 4.7 % on 20k protein
// pairs; 2 is no faster than 0 on DNA.
#ifndef SWGB_KEY_PAIRS
#define SWGB_KEY_PAIRS 1
#endif
// Packed form, boundary-out word: 0 = stored only for columns inside the
// strip (a range check per step); 1 = stored on every step (the words of
// columns outside [0, m) land in ring slots that are overwritten before
// they are flushed, or never flushed).
#ifndef SWGB_BOUT_ANY_COLUMN
#define SWGB_BOUT_ANY_COLUMN 1
#endif
// Packed form with gaps and 32-bit profile words, the row above word 0:
// 0 = two shuffles (the lane above's last word of H and of F) and two
// selects for lane 0; 1 = one shuffle of a word holding both (the boundary
// word's format, which lane 0 takes instead with one select).  Measured
// with the same tuning: +1.1 % on 100k DNA pairs (the byte-profile form
// keeps 0: -0.2 % on 20k protein pairs).
#ifndef SWGB_ONE_SHUFFLE
#define SWGB_ONE_SHUFFLE 1
#endif
// Packed form with 32-bit profile words, the diagonal sum H_diag + s'
// (three terms): 0 = plain adds; 1 = two multiply-adds by a one the
// compiler cannot see, issued on the FMA pipe instead of the ALU pipe.
// Measured: +1.3 % on 100k DNA pairs, +1.5 % together with one shuffle
// (the byte-profile form, one add per word, keeps 0: -0.7 % on protein).
#ifndef SWGB_DADD_FMA
#define SWGB_DADD_FMA 1
#endif
// A lane's R rows as two halves a column apart (2: two independent row
// chains per step) or one block of R rows (1).  Measured on 100k and 200k
// DNA pairs, the split form was 0.2 % and 1.1 % slower, so it is off; it
// stays as a build option (int32 profile only).
template <bool P8, bool PK>
__host__ __device__ constexpr int halves_of() {
    return PK ? 2 : ((SWGB_SPLIT_ROWS && !P8) ? 2 : 1);
}
// blocks between a cp.async and the first use; the copies in flight plus the
// block being read stay within six of the eight 16-byte slots of a ring
template <bool P8, bool PK>
__host__ __device__ constexpr int ahead_of() {
    return unroll_of<P8, PK>() == 4 ? 3 : 2;
}
constexpr int kMaxGroups = 32 >> kMinLog2G;
constexpr int kRingBytes = 128;        // per group and ring

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
// 16 bytes of shared memory into v where p holds (v unchanged elsewhere;
// a predicated load, no branch)
__device__ __forceinline__ void lds16_if(uint4 &v, const uint32_t *ssrc, bool p) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(ssrc);
    asm volatile(
        "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %4, 0;\n\t"
        "@q ld.shared.v4.b32 {%0, %1, %2, %3}, [%5];\n\t}"
        : "+r"(v.x), "+r"(v.y), "+r"(v.z), "+r"(v.w)
        : "r"((int)p), "r"(sa)
        : "memory");
}
// L2 eviction priorities: strip-boundary words stored and read back with
// evict-last, so that they stay in L2 between strips (1; on 100k DNA pairs
// 190 -> 131 MB of DRAM writes per launch, same time), or the default
// policy (0).
#ifndef SWGB_L2_HINTS
#define SWGB_L2_HINTS 1
#endif
__device__ __forceinline__ uint64_t l2_evict_last_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
// cp_async16 issued only where p holds: a predicated instruction, no branch
// (an address formed for a lane with p false is never accessed)
__device__ __forceinline__ void cp_async16_if(void *smem_dst, const void *gsrc, bool p) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile(
        "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %2, 0;\n\t"
        "@q cp.async.cg.shared.global [%0], [%1], 16;\n\t}" ::"r"(d),
        "l"(gsrc), "r"((int)p)
        : "memory");
}
// 16 bytes from shared to global memory where p holds (predicated, no branch)
__device__ __forceinline__ void copy16_s2g_if(uint32_t *gdst, const uint32_t *ssrc, bool p,
                                              uint64_t pol) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(ssrc);
#if SWGB_L2_HINTS
    asm volatile(
        "{\n\t.reg .pred q;\n\t.reg .b32 a, b, c, d;\n\tsetp.ne.b32 q, %2, 0;\n\t"
        "@q ld.shared.v4.b32 {a, b, c, d}, [%1];\n\t"
        "@q st.global.L2::cache_hint.v4.b32 [%0], {a, b, c, d}, %3;\n\t}" ::"l"(gdst),
        "r"(sa), "r"((int)p), "l"(pol)
        : "memory");
#else
    (void)pol;
    asm volatile(
        "{\n\t.reg .pred q;\n\t.reg .b32 a, b, c, d;\n\tsetp.ne.b32 q, %2, 0;\n\t"
        "@q ld.shared.v4.b32 {a, b, c, d}, [%1];\n\t"
        "@q st.global.v4.b32 [%0], {a, b, c, d};\n\t}" ::"l"(gdst),
        "r"(sa), "r"((int)p)
        : "memory");
#endif
}
// Strip-boundary words are read once, by the next strip: once a whole L2
// line of them has landed in shared memory, it is dropped from L2 without a
// write-back (1; the line holds only this buffer's consumed words, 128-byte
// aligned), or left to be written back when evicted (0).  Measured on 100k
// DNA pairs: DRAM traffic per launch 243 -> 105 MB, time unchanged; the
// byte-profile form keeps 0 (3.4 % slower with it on 20k protein pairs).
#ifndef SWGB_DISCARD
#define SWGB_DISCARD 1
#endif
__device__ __forceinline__ void discard_l2_if(const void *line, bool p) {
    asm volatile(
        "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %1, 0;\n\t"
        "@q discard.global.L2 [%0], 128;\n\t}" ::"l"(line), "r"((int)p));
}
// cp_async16_if for boundary words, with the evict-last policy when enabled
__device__ __forceinline__ void cp_async16_bnd_if(void *smem_dst, const void *gsrc, bool p,
                                                  uint64_t pol) {
#if SWGB_L2_HINTS
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile(
        "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %2, 0;\n\t"
        "@q cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %3;\n\t}" ::"r"(d),
        "l"(gsrc), "r"((int)p), "l"(pol)
        : "memory");
#else
    (void)pol;
    cp_async16_if(smem_dst, gsrc, p);
#endif
}


// Sign-extended int8 byte B of w, moved to bits 16..31 (value << 16).
template <int B>
__device__ __forceinline__ int byte_hi(uint32_t w) {
    constexpr uint32_t sel = 0x44u | (uint32_t(B) << 8) | (uint32_t(B | 8) << 12);
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(w), "r"(0u), "r"(sel));
    return (int)d;
}

// prmt.b32 with its sign-replicating selectors (bit 3 of a nibble copies the
// top bit of the selected byte into every bit of the result byte).
__device__ __forceinline__ uint32_t prmt_sx(uint32_t a, uint32_t b, uint32_t sel) {
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
    return d;
}

// Scaled substitution tables, filled once per block: entry x * (A + 1) + c
// is the profile value of row residue x against column residue c, that is
// (s - go) << 16 (int32 profile) or s - go (int8 profile), and entry
// x * (A + 1) + A the pad value.  Two tables: the forward sweep's (rows are
// query residues, s = mat[x][c]) and the transposed reverse sweep's
// (rows are reference residues, s = mat[c][x]).
template <bool P8>
using TabT = typename std::conditional<P8, int8_t, int32_t>::type;

__host__ __device__ constexpr size_t tab_bytes(bool p8, int A) {
    const size_t need = 2 * (size_t)A * (size_t)(A + 1) * (p8 ? 1 : 4);
    return ((need > 1024 ? need : 1024) + 15) & ~(size_t)15;
}

// Profile of the G lanes gb .. gb + G - 1 of one group, filled by all 32
// lanes of the warp together: for column residue c in [0, A] (A = pad) and
// each lane's R rows (rows row_base + t*R .. of the sweep for lane gb + t),
// the table value of the row's residue against c, or the pad value for rows
// past the end.  One work unit is one lane's four rows (an int32 chunk or an
// int8 word) for every c.  Layout [c][chunk][lane]: conflict-free loads
// whatever residue each lane asks for.
template <int R, bool P8, bool PK>
__device__ __forceinline__ void build_profile_group(char *prof, int lane, int gb, int log2g,
                                                    const uint8_t *a, int dir, int row_base,
                                                    int nrows, const TabT<P8> *tab, int A) {
    static_assert(!P8 || R == 8 || R == 16 || R == 32, "int8 profile holds 8, 16 or 32 rows");
    const int G = 1 << log2g;
    const int units = G * (R / 4);
    if (row_base == 0 && dir > 0) {
        // first strip of a forward sweep: the later strips' query rows are
        // read by their profile builds only, one strip at a time; bring the
        // rest of the query (up to 4 KB) into L2 now, so those builds do not
        // wait on DRAM
        const int line = lane * 128 + G * R;
        if (line < nrows && lane * 128 < 4096) {
            const uint8_t *ptr = a + line;
            asm volatile("prefetch.global.L2 [%0];" ::"l"(ptr));
        }
    }
    for (int u = lane; u < units; u += 32) {
        const int tl = u & (G - 1), k = u >> log2g;
        const int tlane = gb + tl;
        int base[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int i = row_base + tl * R + 4 * k + j;
            base[j] = i < nrows ? min((int)a[(ptrdiff_t)i * dir], A - 1) * (A + 1) : -1;
        }
        for (int c = 0; c <= A; ++c) {
            if constexpr (P8) {
                // (packed form with a byte profile: 4 (s - go) in [0, 127], 0
                // past the end)
                uint32_t w = 0u;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int v = base[j] >= 0 ? (int)tab[base[j] + c] : (PK ? 0 : -128);
                    w |= (uint32_t)(uint8_t)(int8_t)v << (8 * j);
                }
                if constexpr (R == 8)
                    *reinterpret_cast<uint32_t *>(prof + ((size_t)c * 32 + tlane) * 8 + k * 4) = w;
                else
                    *reinterpret_cast<uint32_t *>(
                        prof + (((size_t)c * (R / 16) + (k >> 2)) * 32 + tlane) * 16 + (k & 3) * 4) =
                        w;
            } else if constexpr (PK) {
                // packed form: s' = 8 (s - go) >= 0, 0 past the end; the
                // lower R/2 rows go to the high halves
                const int sh = 4 * k >= R / 2 ? 16 : 0;
                int v[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) v[j] = (base[j] >= 0 ? tab[base[j] + c] : 0) << sh;
                *reinterpret_cast<int4 *>(prof + (((size_t)c * (R / 4) + k) * 32 + tlane) * 16) =
                    make_int4(v[0], v[1], v[2], v[3]);
            } else {
                int v[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) v[j] = base[j] >= 0 ? tab[base[j] + c] : kScaledPad;
                *reinterpret_cast<int4 *>(prof + (((size_t)c * (R / 4) + k) * 32 + tlane) * 16) =
                    make_int4(v[0], v[1], v[2], v[3]);
            }
        }
    }
}

template <int R, bool P8>
__device__ __forceinline__ void load_scores(const char *prof, int c, int lane, int (&sc)[R]) {
    if constexpr (P8) {
        uint32_t ws[R / 4];
        if constexpr (R == 8) {
            const uint2 w = *reinterpret_cast<const uint2 *>(prof + ((size_t)c * 32 + lane) * 8);
            ws[0] = w.x;
            ws[1] = w.y;
        } else {
#pragma unroll
            for (int k = 0; k < R / 16; ++k) {
                const uint4 w = *reinterpret_cast<const uint4 *>(
                    prof + (((size_t)c * (R / 16) + k) * 32 + lane) * 16);
                ws[4 * k] = w.x;
                ws[4 * k + 1] = w.y;
                ws[4 * k + 2] = w.z;
                ws[4 * k + 3] = w.w;
            }
        }
#pragma unroll
        for (int k = 0; k < R / 4; ++k) {
            sc[4 * k + 0] = byte_hi<0>(ws[k]);
            sc[4 * k + 1] = byte_hi<1>(ws[k]);
            sc[4 * k + 2] = byte_hi<2>(ws[k]);
            sc[4 * k + 3] = byte_hi<3>(ws[k]);
        }
    } else {
#pragma unroll
        for (int k = 0; k < R / 4; ++k) {
            const int4 v = *reinterpret_cast<const int4 *>(
                prof + (((size_t)c * (R / 4) + k) * 32 + lane) * 16);
            sc[4 * k + 0] = v.x;
            sc[4 * k + 1] = v.y;
            sc[4 * k + 2] = v.z;
            sc[4 * k + 3] = v.w;
        }
    }
}

// Scores of the lane's rows with the upper half of the rows against column
// residue c0 and the lower half against c1 (c0 == c1 for one block of rows).
template <int R, bool P8, int HALVES>
__device__ __forceinline__ void load_scores_halves(const char *prof, int c0, int c1, int lane,
                                                   int (&sc)[R]) {
    if constexpr (HALVES == 1) {
        load_scores<R, P8>(prof, c0, lane, sc);
    } else if constexpr (P8) {
        static_assert(R == 16, "split int8 profile rows assume 16 rows per lane");
        const uint2 w0 = *reinterpret_cast<const uint2 *>(prof + ((size_t)c0 * 32 + lane) * 16);
        const uint2 w1 = *reinterpret_cast<const uint2 *>(prof + ((size_t)c1 * 32 + lane) * 16 + 8);
        const uint32_t ws[4] = {w0.x, w0.y, w1.x, w1.y};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            sc[4 * k + 0] = byte_hi<0>(ws[k]);
            sc[4 * k + 1] = byte_hi<1>(ws[k]);
            sc[4 * k + 2] = byte_hi<2>(ws[k]);
            sc[4 * k + 3] = byte_hi<3>(ws[k]);
        }
    } else {
        static_assert(R % 8 == 0, "split int32 profile rows need whole 4-row chunks per half");
#pragma unroll
        for (int k = 0; k < R / 4; ++k) {
            const int c = k < R / 8 ? c0 : c1;
            const int4 v = *reinterpret_cast<const int4 *>(
                prof + (((size_t)c * (R / 4) + k) * 32 + lane) * 16);
            sc[4 * k + 0] = v.x;
            sc[4 * k + 1] = v.y;
            sc[4 * k + 2] = v.z;
            sc[4 * k + 3] = v.w;
        }
    }
}

// Per-lane bookkeeping of a group that only the strip and sweep transitions
// read: kept in shared memory (one array per field, indexed by thread) so
// the step loop's registers hold the DP state alone.
struct Cold {
    const uint8_t **a;   // row residues of the current sweep (a[i * dir])
    uint32_t **bnd;      // the pair's strip-boundary words
    int *n, *m, *passes, *ps, *target, *id, *S, *qend, *rend, *best_row;
    uint32_t *best_key;
};

constexpr int kColdWords = 2 * 2 + 11;  // 32-bit words per lane

}  // namespace

template <int R, bool P8, bool LIN, bool PK>
__global__ void __launch_bounds__(kGroupWarps * 32, (PK && R > 16) ? 2 : kGroupMinBlocks)
    sw_group_kernel(const __grid_constant__ GroupParams p) {
    static_assert(!PK || R % 16 == 0, "the packed form holds 16 rows per 8 words");
    static_assert(!(PK && P8) || R == 16, "the packed byte profile holds 16 rows per lane");
    extern __shared__ __align__(16) char smem_group[];
    constexpr int kHalves = halves_of<P8, PK>();
    constexpr int W = R / 2;  // packed words per lane
    // packed form: scores scaled by SC, leaving CB low bits for the row code
    // of an end-key chain of CL words (32-bit profile words: 8 / 3 / 8; byte
    // profile: 4 / 2 / 4, so that 4 (s - go) fits a byte)
    constexpr int SC = P8 ? 4 : 8;
    constexpr int CB = P8 ? 2 : 3;
    constexpr int CL = 1 << CB;
    constexpr int NC = W / CL;  // end-key chains
    constexpr int kU = unroll_of<P8, PK>();
    constexpr int kAhead = ahead_of<P8, PK>();
    static_assert(kU == 4 || kU == 8, "blocks move whole 16-byte chunks of 4 boundary columns");
    const int A = p.alphabet;
    const int go = p.gap_open, ge = p.gap_extend;
    const int goS = go * 65536, geS = ge * 65536;
    // packed form: SC ge and SC go in both halves
    const uint32_t geP = ((uint32_t)(SC * ge) & 0xFFFFu) * 0x10001u;
    const uint32_t goP = ((uint32_t)(SC * go) & 0xFFFFu) * 0x10001u;
    // boundary word of "no row above": H = 0 (stored as H + go) and F = -inf
    // (0xC000 = -16384 in the high half, -2^30 scaled); packed form: H = 0 and
    // F = go (F - go = 0), which gives the row below the same values
    const uint32_t kNoBound = PK ? 0u : (0xC0000000u | ((uint32_t)go & 0xFFFFu));
    constexpr int NT = kGroupWarps * 32;
    // 1 (blocks have NT threads), unknown to the compiler
    [[maybe_unused]] const uint32_t one_opaque = blockDim.x / NT;
    const int t = threadIdx.x;
    const int warp = t >> 5, lane = t & 31;
    const uint64_t l2pol = SWGB_L2_HINTS ? l2_evict_last_policy() : 0ull;
    const size_t prof_bytes = P8 ? (size_t)(A + 1) * 32 * R : (size_t)(A + 1) * (R / 4) * 32 * 16;
    // shared memory: rings (16-byte aligned) | score tables | cold state | profiles
    char *rings = smem_group + (size_t)warp * 3 * kMaxGroups * kRingBytes;
    TabT<P8> *tab_fwd = reinterpret_cast<TabT<P8> *>(smem_group + (size_t)kGroupWarps * 3 *
                                                                      kMaxGroups * kRingBytes);
    TabT<P8> *tab_rev = tab_fwd + A * (A + 1);
    char *cold_base = reinterpret_cast<char *>(tab_fwd) + tab_bytes(P8, A);
    char *prof = cold_base + (size_t)kColdWords * 4 * NT + warp * prof_bytes;
    Cold cold;
    cold.a = reinterpret_cast<const uint8_t **>(cold_base);
    cold.bnd = reinterpret_cast<uint32_t **>(cold_base + 8 * NT);
    int *cw = reinterpret_cast<int *>(cold_base + 16 * NT);
    cold.n = cw;
    cold.m = cw + NT;
    cold.passes = cw + 2 * NT;
    cold.ps = cw + 3 * NT;
    cold.target = cw + 4 * NT;
    cold.id = cw + 5 * NT;
    cold.S = cw + 6 * NT;
    cold.qend = cw + 7 * NT;
    cold.rend = cw + 8 * NT;
    cold.best_row = cw + 9 * NT;
    cold.best_key = reinterpret_cast<uint32_t *>(cw + 10 * NT);
    {
        // a launch whose queues are all empty (a route of a device-planned
        // batch with no pairs on it) ends before any setup
        int queued = 0;
        for (int c = 0; c < p.n_classes; ++c) queued += p.classes[c].count;
        if (queued == 0) return;
    }
    for (int i = t; i < A * (A + 1); i += blockDim.x) {
        const int x = i / (A + 1), c = i - x * (A + 1);
        if (c == A) {
            tab_fwd[i] = (TabT<P8>)(PK ? 0 : P8 ? -128 : kScaledPad);
            tab_rev[i] = (TabT<P8>)(PK ? 0 : P8 ? -128 : kScaledPad);
        } else {
            // the plan takes the int8 profile only when s - go fits in int8
            const int vf = (int)p.mat[x * A + c] - go, vr = (int)p.mat[c * A + x] - go;
            tab_fwd[i] = (TabT<P8>)(PK ? SC * vf : P8 ? vf : vf * 65536);
            tab_rev[i] = (TabT<P8>)(PK ? SC * vr : P8 ? vr : vr * 65536);
        }
    }
    __syncthreads();

    // this warp starts on the class whose warp range holds it, then walks
    // the classes cyclically
    const int wid = blockIdx.x * kGroupWarps + warp;
    int start = 0;
    for (int c = 1; c < p.n_classes; ++c)
        if (wid >= p.classes[c].warp_begin) start = c;
    for (int visit = 0; visit < p.n_classes; ++visit) {
        const int cls = (start + visit) % p.n_classes;
        const ClassInfo ci = p.classes[cls];
        const int log2g = ci.log2g;
        const int G = 1 << log2g;
        const int gl = lane & (G - 1);
        const int gbase = lane & ~(G - 1);
        const int gid = lane >> log2g;
        // packed form: the halves of word 0's row above (lane 0 takes the
        // boundary word's low half, the others the high half of a shuffle)
        const uint32_t selH = gl == 0 ? 0x5410u : 0x5432u;
        const unsigned gmask = G == 32 ? kFull : (((1u << G) - 1u) << gbase);
        uint8_t *res_ring = reinterpret_cast<uint8_t *>(rings) + gid * kRingBytes;
        uint32_t *bin_ring =
            reinterpret_cast<uint32_t *>(rings + kMaxGroups * kRingBytes + gid * kRingBytes);
        uint32_t *bout_ring =
            reinterpret_cast<uint32_t *>(rings + 2 * kMaxGroups * kRingBytes + gid * kRingBytes);

        // hot state: DP registers, the strip's step counters and stream cursors
        int H[R], E[R];
        uint32_t K[R];
        int diag0 = goS, outH = goS, outF = kScaledNegInf;
        // split rows: the upper half's last row (H + go and F) at the lower
        // half's column (from the previous step) and one column earlier, and
        // the column residue the lower half takes next
        int midH = goS, midF = kScaledNegInf, midD = goS, ccarry = A;
        // packed form: the lane's words, its last word and that word's F of
        // the step before, word 0's row above of the step before, and the
        // end tracking (threshold, its "keep the score" mask, one record per
        // half: column << 16 | 8 score + row code)
        uint32_t Hw[W], Ew[W];
        uint32_t outHw = 0u, outFw = 0u, diag0w = 0u, outX = 0u;
        uint32_t Tw[NC], rec_lo[NC], rec_hi[NC], tmask = (CL - 1) * 0x10001u;
#pragma unroll
        for (int c = 0; c < NC; ++c) Tw[c] = (CL - 1) * 0x10001u, rec_lo[c] = rec_hi[c] = 0u;
        int s = 0, lim = 0, stop = 0, dir = 1;
        const uint8_t *bcol = p.r;  // column 0 of the current sweep
        int roff = 0;               // bcol's offset in its 16-byte chunk (mirrored if dir < 0)
        int rc_next = 0, rc_last = -1;  // next residue chunk to fetch, last useful one
        int bi_next = 0, bi_last = -1;  // same for boundary-in chunks (4 words each)
        int bo_done = 0;                // boundary-out words written so far
        const uint32_t *bin = p.scratch;
        uint32_t *bout = p.scratch;
        // next 128-byte line of boundary-in words to drop from L2
        [[maybe_unused]] const uint32_t *bdisc = p.scratch;
        bool has_in = false, has_out = false;
        bool live = false, rev = false, drained = false;
        bool need_prof = false;  // this lane's group started a strip without its profile
#pragma unroll
        for (int r = 0; r < R; ++r) {
            H[r] = goS;
            E[r] = kScaledNegInf;
            K[r] = 0u;
        }
#pragma unroll
        for (int k = 0; k < W; ++k) Hw[k] = Ew[k] = 0u;
        cold.id[t] = -1;

        // Issues the cp.async copies that are due: residue chunks up to the
        // one holding column `upto`, boundary-in chunks up to column `upto`.
        // Only lane 0 of a group copies; every lane keeps the cursors.
        auto fetch_ahead = [&](int upto) {
            const int rc_want = min((roff + upto) >> 4, rc_last);
            while (rc_next <= rc_want) {
                if (gl == 0) {
                    const uint8_t *base =
                        reinterpret_cast<const uint8_t *>((uintptr_t)bcol & ~(uintptr_t)15);
                    const uint8_t *src = base + (ptrdiff_t)(dir > 0 ? rc_next : -rc_next) * 16;
                    cp_async16(res_ring + (((uintptr_t)src >> 4) & 7) * 16, src);
                }
                ++rc_next;
            }
            const int bi_want = min(upto >> 2, bi_last);
            while (bi_next <= bi_want) {
                if (gl == 0) cp_async16(bin_ring + (bi_next & 7) * 4, bin + bi_next * 4);
                ++bi_next;
            }
        };
        // The copies due in a steady-state block (columns advance by kU < 16
        // per block: at most one residue chunk and kU / 4 boundary chunks),
        // as predicated instructions: the groups of a warp are at different
        // columns of different pairs, so per-group branches here diverged on
        // every block (a branch-free block measured 11 % faster on 100k and
        // 200k DNA pairs, 6 % on 20k protein pairs).
        auto fetch_block = [&](int upto) {
            const int rc_want = min((roff + upto) >> 4, rc_last);
            const bool r_due = rc_next <= rc_want;
            const uint8_t *base = reinterpret_cast<const uint8_t *>((uintptr_t)bcol & ~(uintptr_t)15);
            const uint8_t *src = base + (ptrdiff_t)(dir > 0 ? rc_next : -rc_next) * 16;
            cp_async16_if(res_ring + (((uintptr_t)src >> 4) & 7) * 16, src, r_due && gl == 0);
            rc_next += r_due ? 1 : 0;
            const int bi_want = min(upto >> 2, bi_last);
#pragma unroll
            for (int k = 0; k < kU / 4; ++k) {
                const bool b_due = bi_next <= bi_want;
                cp_async16_bnd_if(bin_ring + (bi_next & 7) * 4, bin + bi_next * 4,
                                  b_due && gl == 0, l2pol);
                bi_next += b_due ? 1 : 0;
            }
        };
        auto flush_block = [&](int upto) {
#pragma unroll
            for (int k = 0; k < kU / 4; ++k) {
                const bool due = bo_done < upto;
                copy16_s2g_if(bout + bo_done, bout_ring + (bo_done & 31), due && gl == G - 1,
                              l2pol);
                bo_done += due ? 4 : 0;
            }
        };
        // Writes boundary-out words [bo_done, upto) (whole 4-word groups,
        // upto a multiple of 4) from the ring to global memory (strip ends).
        auto flush_out = [&](int upto) {
            while (bo_done < upto) {
                if (gl == G - 1)
                    *reinterpret_cast<uint4 *>(bout + bo_done) =
                        *reinterpret_cast<const uint4 *>(bout_ring + (bo_done & 31));
                bo_done += 4;
            }
        };
        // Starts strip ps of the current sweep: profile of this lane's rows,
        // fresh DP state, stream cursors; waits for the strip's first data.
        auto begin_strip = [&](int ps) {
            const int n = cold.n[t], m = cold.m[t];
            need_prof = true;  // filled by the whole warp before the next block
#pragma unroll
            for (int r = 0; r < R; ++r) {
                H[r] = goS;
                E[r] = kScaledNegInf;
                K[r] = 0u;
            }
            diag0 = goS;
            outH = goS;
            outF = kScaledNegInf;
            midH = goS;
            midF = kScaledNegInf;
            midD = goS;
            ccarry = A;
            if constexpr (PK) {
#pragma unroll
                for (int k = 0; k < W; ++k) Hw[k] = Ew[k] = 0u;
                outHw = outFw = diag0w = outX = 0u;
                // forward: best score 0 with the largest row code; reverse:
                // just below the score S with any row code
                const uint32_t t0 = rev ? (uint32_t)(SC * cold.target[t] - 1) : (uint32_t)(CL - 1);
                tmask = rev ? 0u : (CL - 1) * 0x10001u;
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    Tw[c] = (t0 & 0xFFFFu) * 0x10001u;
                    rec_lo[c] = rec_hi[c] = 0u;
                }
            }
            s = 0;
            // the lane's last row reaches the last column kHalves * G - 1 steps late
            lim = stop + kHalves * G - 1;
            const int m4 = (m + 3) & ~3;
            uint32_t *bnd = cold.bnd[t];
            bin = bnd + ((ps + 1) & 1) * m4;
            bout = bnd + (ps & 1) * m4;
            bdisc = reinterpret_cast<const uint32_t *>(((uintptr_t)bin + 127) & ~(uintptr_t)127);
            has_in = ps > 0;
            has_out = ps + 1 < cold.passes[t];
            rc_next = 0;
            bi_next = 0;
            bi_last = has_in ? (stop - 1) >> 2 : -1;
            bo_done = 0;
            cold.ps[t] = ps;
            {
                // the strip's row residues, read by the profile build at the
                // next block: ask for this lane's rows now, so the build hits
                // L1 (+1.2 % on 20k protein pairs, +0.1-0.3 % on DNA)
                const int row = ps * G * R + gl * R;
                if (row < n) {
                    const uint8_t *ptr = cold.a[t] + (ptrdiff_t)row * dir;
                    asm volatile("prefetch.global.L1 [%0];" ::"l"(ptr));
                }
            }
            fetch_ahead(kAhead * kU + kU - 1);
            cp_async_commit();
            cp_async_wait<0>();
            __syncwarp(gmask);
        };
        // Starts a sweep over (a, n) x (b, m) in direction d.
        auto begin_sweep = [&](const uint8_t *a, const uint8_t *b, int n, int m, int d) {
            cold.a[t] = a;
            bcol = b;
            dir = d;
            cold.n[t] = n;
            cold.m[t] = m;
            const int passes = (n > 0 && m > 0) ? (n + G * R - 1) / (G * R) : 0;
            cold.passes[t] = passes;
            cold.best_key[t] = 0u;
            cold.best_row[t] = 0x7fffffff;
            const int b15 = (int)((uintptr_t)b & 15);
            roff = d > 0 ? b15 : 15 - b15;
            rc_last = m > 0 ? (roff + m - 1) >> 4 : -1;
            if (passes > 0) {
                stop = m;
                begin_strip(0);
            } else {
                stop = 0;
                s = 0;
                lim = 0;
                has_in = has_out = false;
                bi_last = -1;
                cold.ps[t] = 0;
            }
        };

        for (;;) {
            // ---- idle groups take the next pair of the class
            if (!live && !drained) {
                int idx = 0;
                if (gl == 0) idx = atomicAdd(p.counters + cls, 1);
                idx = __shfl_sync(gmask, idx, gbase);
                if (idx >= ci.count) {
                    drained = true;
                } else {
                    const PairInfo pi = p.pairs[ci.first + idx];
                    live = true;
                    rev = false;
                    cold.id[t] = pi.id;
                    cold.bnd[t] =
                        p.scratch + (p.slot_words > 0
                                         ? ((size_t)wid * 32 + gbase) * (size_t)p.slot_words
                                         : (size_t)(pi.scratch >= 0 ? pi.scratch : 0));
                    begin_sweep(p.q + pi.q, p.r + pi.r, pi.n, pi.m, 1);
                }
            }
            if (__all_sync(kFull, !live)) break;  // every group drained and idle

            // ---- profiles of the groups that started a strip, built by all lanes
            unsigned need = __ballot_sync(kFull, need_prof);
            if (need) {
                __syncwarp();  // the groups' sweep state in shared memory is visible
                while (need) {
                    const int gb = (__ffs(need) - 1) & ~(G - 1);
                    const int tg = warp * 32 + gb;
                    const int gdir = __shfl_sync(kFull, dir, gb);
                    const bool grev = __shfl_sync(kFull, (int)rev, gb) != 0;
                    build_profile_group<R, P8, PK>(prof, lane, gb, log2g, cold.a[tg], gdir,
                                               cold.ps[tg] * G * R, cold.n[tg],
                                               grev ? tab_rev : tab_fwd, A);
                    need &= G == 32 ? 0u : ~(((1u << G) - 1u) << gb);
                }
                __syncwarp();
                need_prof = false;
            }

            const int mcols = live ? stop : 0;

            // ---- staging: copies for kAhead blocks ahead, then wait for this block's
            fetch_block(s + kAhead * kU + kU - 1);
            cp_async_commit();
            cp_async_wait<kAhead>();
            __syncwarp();
#if SWGB_DISCARD
            if constexpr (!P8) {
                // the boundary-in words of columns below s + kU are in the ring
                const bool dd = gl == 0 && live && has_in && bdisc + 32 <= bin + min(s + kU, stop);
                discard_l2_if(bdisc, dd);
                bdisc += dd ? 32 : 0;
            }
#endif

            // column residues of the upper rows (the lower half takes each one
            // step later, so its residue is the upper half's of the step before)
            int cres[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int j = s + u - kHalves * gl;
                const bool in = (unsigned)j < (unsigned)mcols;
                const int byte = res_ring[((uint32_t)(uintptr_t)bcol + j * dir) & (kRingBytes - 1)];
                cres[u] = in ? min(byte, A - 1) : A;
            }
            uint32_t bws[kU];
#pragma unroll
            for (int h = 0; h < kU / 4; ++h) {
                uint4 bw = make_uint4(kNoBound, kNoBound, kNoBound, kNoBound);
                if constexpr (PK || !P8) {
                    // predicated load, no branch (+1.3 % on 100k DNA pairs)
                    lds16_if(bw, bin_ring + (((s >> 2) + h) & 7) * 4,
                             gl == 0 && has_in && s + 4 * h < mcols);
                } else if (gl == 0 && has_in && s + 4 * h < mcols) {
                    // (the int8-profile int32 form keeps the branch: the
                    // predicated form's registers spill there)
                    bw = *reinterpret_cast<const uint4 *>(bin_ring + (((s >> 2) + h) & 7) * 4);
                }
                bws[4 * h] = bw.x;
                bws[4 * h + 1] = bw.y;
                bws[4 * h + 2] = bw.z;
                bws[4 * h + 3] = bw.w;
            }

            // ---- U wavefront steps, the same instructions on every lane.  With
            // split rows, rows [0, R/2) work on column j0 = s - 2 gl and rows
            // [R/2, R) on j0 - 1: two independent row chains per step, the
            // lower one fed by the upper one's last row of the step before.
            // packed form: this block's first step in both halves (s < 2^16)
            const uint32_t stw0 = (uint32_t)s * 0x10001u;
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                if constexpr (PK) {
                    // packed: low halves rows [0, R/2) at column j0 = s - 2 gl,
                    // high halves rows [R/2, R) at j0 - 1
                    const int j0 = s + u - 2 * gl;
                    const int j1 = j0 - 1;
                    const bool in1 = (unsigned)j1 < (unsigned)mcols;
                    uint32_t upH, upF;
                    if constexpr (SWGB_ONE_SHUFFLE && !LIN && !P8) {
                        // the lane above's last row as one word (H low, F - go
                        // high); lane 0: the previous strip's boundary word
                        uint32_t inX = __shfl_up_sync(kFull, outX, 1, G);
                        if (gl == 0) inX = bws[u];
                        upH = __byte_perm(inX, outHw, 0x5410);
                        upF = __byte_perm(inX, outFw, 0x5432);
                    } else {
                        uint32_t inH = __shfl_up_sync(kFull, outHw, 1, G);
                        uint32_t inF = LIN ? 0u : __shfl_up_sync(kFull, outFw, 1, G);
                        if (gl == 0) {
                            // previous strip's last row (H low, F - go high), or (0, 0)
                            inH = bws[u];
                            inF = bws[u];
                        }
                        // word 0's row above: the lane above's last row (high half of
                        // its last word; lane 0: the boundary word's halves) and this
                        // lane's row R/2 - 1 of the step before
                        upH = __byte_perm(inH, outHw, selH);
                        upF = LIN ? 0u : __byte_perm(inF, outFw, 0x5432);
                    }
                    int c0 = cres[u];
                    int c1 = u == 0 ? ccarry : cres[u - 1];
#if SWGB_STEP_ORDER_FENCE
                    asm volatile("" : "+r"(c0), "+r"(c1) : "r"(upH));
#endif
                    // s' of word k: 32-bit profile, the sum of a low-half word
                    // (row k, column j0) and a high-half word (row R/2 + k,
                    // column j1); byte profile, the two rows' bytes moved to
                    // the halves (zero-extended: every byte is below 128)
                    uint32_t scw[W];
                    [[maybe_unused]] uint32_t sch[W];
                    if constexpr (P8) {
                        const uint2 b0 = *reinterpret_cast<const uint2 *>(
                            prof + ((size_t)c0 * 32 + lane) * 16);
                        const uint2 b1 = *reinterpret_cast<const uint2 *>(
                            prof + ((size_t)c1 * 32 + lane) * 16 + 8);
#pragma unroll
                        for (int k = 0; k < W; ++k) {
                            constexpr unsigned kSel[4] = {0xC480u, 0xD591u, 0xE6A2u, 0xF7B3u};
                            scw[k] = prmt_sx(k < 4 ? b0.x : b0.y, k < 4 ? b1.x : b1.y, kSel[k & 3]);
                        }
                    } else {
                        int sc[R];
                        load_scores_halves<R, false, 2>(prof, c0, c1, lane, sc);
#pragma unroll
                        for (int k = 0; k < W; ++k) {
                            if constexpr (SWGB_DADD_FMA != 0) {
                                scw[k] = (uint32_t)sc[k];
                                sch[k] = (uint32_t)sc[W + k];
                            } else {
                                scw[k] = (uint32_t)sc[k] + (uint32_t)sc[W + k];
                            }
                        }
                    }
                    uint32_t diag = diag0w;
                    uint32_t F = LIN ? 0u : __viaddmax_s16x2(upF, geP, upH);
                    uint32_t hprev = upH;
                    uint32_t acc[NC];
                    uint32_t hc_even = 0u;  // h + row code of the pair's first word
#pragma unroll
                    for (int c = 0; c < NC; ++c) acc[c] = Tw[c];
#pragma unroll
                    for (int k = 0; k < W; ++k) {
                        // carry-free: both halves of every term are non-negative
                        uint32_t D;
                        if constexpr (SWGB_DADD_FMA && !P8) {
                            asm("mad.lo.u32 %0, %1, %2, %3;"
                                : "=r"(D) : "r"(scw[k]), "r"(one_opaque), "r"(diag));
                            {
                                uint32_t D2;
                                asm("mad.lo.u32 %0, %1, %2, %3;"
                                    : "=r"(D2) : "r"(sch[k]), "r"(one_opaque), "r"(D));
                                D = D2;
                            }
                        } else {
                            D = diag + scw[k];
                        }
                        uint32_t V;
                        if constexpr (LIN) {
                            // go == ge: E - go = H_left and F - go = H_up exactly
                            V = __vimax3_s16x2(D, Hw[k], hprev);
                        } else {
                            if (k > 0) F = __viaddmax_s16x2(F, geP, hprev);
                            Ew[k] = __viaddmax_s16x2(Ew[k], geP, Hw[k]);
                            V = __vimax3_s16x2(D, Ew[k], F);
                        }
                        const uint32_t h = __viaddmax_s16x2_relu(V, goP, 0u);
                        diag = Hw[k];
                        Hw[k] = h;
                        hprev = h;
                        const uint32_t code = (uint32_t)(CL - 1 - k % CL) * 0x10001u;
                        if constexpr (SWGB_KEY_PAIRS == 0) {
                            acc[k / CL] = __viaddmax_s16x2(h, code, acc[k / CL]);
                        } else {
                            // the low CB bits of both halves of h are 0 and the
                            // code is below 2^CB, so the 32-bit add is per half
                            uint32_t hc;
                            if constexpr (SWGB_KEY_PAIRS == 2)
                                asm("mad.lo.u32 %0, %1, %2, %3;"
                                    : "=r"(hc) : "r"(h), "r"(one_opaque), "r"(code));
                            else
                                hc = h + code;
                            if (k & 1)
                                acc[k / CL] = __vimax3_s16x2(hc_even, hc, acc[k / CL]);
                            else
                                hc_even = hc;
                        }
                    }
                    outHw = hprev;
                    outFw = F;
                    outX = __byte_perm(outHw, outFw, 0x7632);
                    if (gl == G - 1 && has_out && (SWGB_BOUT_ANY_COLUMN || in1))
                        bout_ring[j1 & 31] = outX;
                    diag0w = upH;
                    // a half whose best score grew records (step, acc half); the
                    // step gives the column: j0 = step - 2 gl, j1 = j0 - 1
                    // (acc >= Tw in both halves; "Tw >= acc" means unchanged)
                    const uint32_t stw = stw0 + (uint32_t)u * 0x10001u;
#pragma unroll
                    for (int c = 0; c < NC; ++c) {
                        bool keep_hi, keep_lo;
                        (void)__vibmax_s16x2(Tw[c], acc[c], &keep_hi, &keep_lo);
                        if (!keep_lo) rec_lo[c] = __byte_perm(acc[c], stw, 0x5410);
                        if (!keep_hi) rec_hi[c] = __byte_perm(acc[c], stw, 0x7632);
                        Tw[c] = acc[c] | tmask;
                    }
                } else {
                    constexpr int RH = R / kHalves;
                    const int j0 = s + u - kHalves * gl;  // column of the upper rows
                    const int j1 = j0 - (kHalves - 1);    // column of the lane's last row
                    const bool in1 = (unsigned)j1 < (unsigned)mcols;
                    int inH = __shfl_up_sync(kFull, outH, 1, G);
                    int inF = LIN ? 0 : __shfl_up_sync(kFull, outF, 1, G);
                    if (gl == 0) {
                        // previous strip's last row, or H = 0 / F = -inf above the
                        // first strip and outside the columns
                        const uint32_t w = bws[u];
                        inH = (int)(w << 16);
                        inF = (int)(w & 0xFFFF0000u);
                    }
                    int c0 = cres[u];
                    int c1 = kHalves == 2 ? (u == 0 ? ccarry : cres[u - 1]) : c0;
    #if SWGB_STEP_ORDER_FENCE
                    // keep this step's profile loads after its shuffle, so the
                    // compiler does not hoist every unrolled step's loads
                    asm volatile("" : "+r"(c0), "+r"(c1) : "r"(inH));
    #endif
                    int sc[R];
                    load_scores_halves<R, P8, kHalves>(prof, c0, c1, lane, sc);
                    // key column part, less go: the key of H + go is (H << 16) + cj
                    const int cjg0 = kColBase - j0 - goS;
                    // upper rows, from the row above (shuffle or strip boundary)
                    int diag = diag0;
                    int F = LIN ? 0 : __viaddmax_s32(inF, geS, inH);
                    int hprev = inH;
    #pragma unroll
                    for (int r = 0; r < RH; ++r) {
                        int h;
                        if constexpr (LIN) {
                            // go == ge: E = H_left + go and F = H_up + go exactly
                            h = __vimax3_s32_relu(diag + sc[r], H[r], hprev) + goS;
                        } else {
                            if (r > 0) F = __viaddmax_s32(F, geS, hprev);
                            E[r] = __viaddmax_s32(E[r], geS, H[r]);
                            h = __vimax3_s32_relu(diag + sc[r], E[r], F) + goS;
                        }
                        diag = H[r];
                        H[r] = h;
                        hprev = h;
                        K[r] = (uint32_t)__viaddmax_s32(h, cjg0, (int)K[r]);
                    }
                    if constexpr (kHalves == 2) {
                        // lower rows, one column behind, from the upper half's last
                        // row of the previous step
                        const int upH = hprev, upF = F;
                        const int cjg1 = cjg0 + 1;
                        int diag1 = midD;
                        int F1 = LIN ? 0 : __viaddmax_s32(midF, geS, midH);
                        int hprev1 = midH;
    #pragma unroll
                        for (int r = RH; r < R; ++r) {
                            int h;
                            if constexpr (LIN) {
                                h = __vimax3_s32_relu(diag1 + sc[r], H[r], hprev1) + goS;
                            } else {
                                if (r > RH) F1 = __viaddmax_s32(F1, geS, hprev1);
                                E[r] = __viaddmax_s32(E[r], geS, H[r]);
                                h = __vimax3_s32_relu(diag1 + sc[r], E[r], F1) + goS;
                            }
                            diag1 = H[r];
                            H[r] = h;
                            hprev1 = h;
                            K[r] = (uint32_t)__viaddmax_s32(h, cjg1, (int)K[r]);
                        }
                        midD = midH;
                        midH = upH;
                        midF = upF;
                        hprev = hprev1;
                        F = F1;
                    }
                    outH = hprev;
                    outF = F;
                    if (gl == G - 1 && has_out && in1)
                        bout_ring[j1 & 31] = __byte_perm((uint32_t)outH, (uint32_t)outF, 0x7632);
                    diag0 = inH;
                }
            }
            ccarry = cres[kU - 1];
            s += kU;
            // words of the columns below s - kHalves * G + 1 are complete; the
            // 4-word group holding the last column waits for the strip end
            flush_block(has_out ? min((s - kHalves * G + 1) & ~3, mcols & ~3) : 0);

            // ---- end of a strip / sweep
            if (live && s >= lim) {
                if (has_out) {
                    // the next strip reads whole 4-word groups without a column
                    // check: the columns past the last one say "no row above"
                    if (gl == G - 1)
                        for (int c = mcols; c < ((mcols + 3) & ~3); ++c) bout_ring[c & 31] = kNoBound;
                    flush_out((mcols + 3) & ~3);
                }
                const int ps = cold.ps[t], passes = cold.passes[t];
                const int row0 = ps * G * R + gl * R;
                uint32_t best_key = cold.best_key[t];
                int best_row = cold.best_row[t];
                // reverse sweep: this strip's smallest row holding a cell of the
                // forward score, with that row's smallest such column
                int frow = 0x7fffffff, fcol = 0;
                if (!rev) {
                    if (ps < passes) {
                        if constexpr (PK) {
                            // the records of both halves and every chain, in
                            // ascending row order (ties keep the smaller row)
#pragma unroll
                            for (int q = 0; q < 2 * NC; ++q) {
                                const int hh = q / NC, c = q % NC;
                                const uint32_t rec = hh ? rec_hi[c] : rec_lo[c];
                                const int val = (int)(rec & 0xFFFFu);
                                const int col = min((int)(rec >> 16) - 2 * gl - hh, kColBase);
                                const uint32_t key =
                                    ((uint32_t)(val >> CB) << 16) | (uint32_t)(kColBase - col);
                                const int row = row0 + hh * W + CL * c + (CL - 1) - (val & (CL - 1));
                                if ((val >> CB) > 0 && key > best_key) {
                                    best_key = key;
                                    best_row = row;
                                }
                            }
                        } else {
#pragma unroll
                            for (int r = 0; r < R; ++r)
                                if (K[r] > best_key) {
                                    best_key = K[r];
                                    best_row = row0 + r;
                                }
                        }
                    }
                    cold.best_key[t] = best_key;
                    cold.best_row[t] = best_row;
                } else {
                    const int target = cold.target[t];
                    if constexpr (PK) {
                        // descending row order, so that the smallest row's
                        // record is the one kept
#pragma unroll
                        for (int q = 2 * NC - 1; q >= 0; --q) {
                            const int hh = q / NC, c = q % NC;
                            const uint32_t rec = hh ? rec_hi[c] : rec_lo[c];
                            const int val = (int)(rec & 0xFFFFu);
                            if ((val >> CB) >= target) {
                                frow = row0 + hh * W + CL * c + (CL - 1) - (val & (CL - 1));
                                fcol = (int)(rec >> 16) - 2 * gl - hh;
                            }
                        }
                    } else {
#pragma unroll
                        for (int r = R - 1; r >= 0; --r)
                            if ((int)(K[r] >> 16) >= target) {
                                frow = row0 + r;
                                fcol = kColBase - (int)(K[r] & 0xFFFFu);
                            }
                    }
                    for (int off = 1; off < G; off <<= 1) {
                        const int orow = __shfl_xor_sync(gmask, frow, off, G);
                        const int ocol = __shfl_xor_sync(gmask, fcol, off, G);
                        if (orow < frow) {
                            frow = orow;
                            fcol = ocol;
                        }
                    }
                }
                // boundary words stored by lane G-1 are read by lane 0's copies
                // of the next strip; both lanes are in this warp, so a
                // block-scope fence and the warp barrier below order the
                // stores before those copies (a device-scope fence measured
                // 0.6 % slower)
                if (has_out) __threadfence_block();
                cp_async_wait<0>();
                __syncwarp(gmask);
                const bool rev_found = rev && frow != 0x7fffffff;
                if (ps + 1 < passes && !rev_found) {
                    begin_strip(ps + 1);
                } else {
                    bool done = true;
                    if (!rev) {
                        for (int off = 1; off < G; off <<= 1) {
                            const uint32_t ok = __shfl_xor_sync(gmask, best_key, off, G);
                            const int orow = __shfl_xor_sync(gmask, best_row, off, G);
                            if (ok > best_key || (ok == best_key && orow < best_row)) {
                                best_key = ok;
                                best_row = orow;
                            }
                        }
                        const int S = (int)(best_key >> 16);
                        const int qend = best_row;
                        const int rend = kColBase - (int)(best_key & 0xFFFFu);
                        cold.S[t] = S;
                        if (S > 0) {
                            cold.qend[t] = qend;
                            cold.rend[t] = rend;
                        }
                        if (S > 0 && !p.ends_only) {
                            cold.target[t] = S;
                            rev = true;
                            done = false;
                            // transposed: reversed reference prefix as rows,
                            // reversed query prefix as columns
                            begin_sweep(bcol + rend, cold.a[t] + qend, rend + 1, qend + 1, -1);
                        }
                    }
                    if (done) {
                        if (gl == 0) {
                            const int S = cold.S[t];
                            const int id = cold.id[t];
                            int o0 = 0, o1 = -1, o2 = -1, o3 = -1, o4 = -1;
                            if (S > 0) {
                                const int qend = cold.qend[t], rend = cold.rend[t];
                                if (!rev_found && !p.ends_only)
                                    atomicOr(p.status, kStatusReverseMismatch);
                                o0 = S;
                                o1 = qend;
                                o2 = rend;
                                o3 = rev_found ? qend - fcol : -1;
                                o4 = rev_found ? rend - frow : -1;
                            }
                            p.out.score[id] = o0;
                            p.out.qend[id] = o1;
                            p.out.rend[id] = o2;
                            if (!p.ends_only) {
                                p.out.qstart[id] = o3;
                                p.out.rstart[id] = o4;
                            }
                        }
                        live = false;
                        rev = false;
                        stop = 0;
                        has_in = has_out = false;
                        rc_last = -1;
                        bi_last = -1;
                        __syncwarp(gmask);
                    }
                }
            }
        }
        cp_async_wait<0>();
        __syncwarp();
    }
}

size_t group_smem_bytes(ProfileKind kind, int alphabet) {
    const size_t rows = (size_t)rows_of(kind);
    const bool bytes = kind == ProfileKind::kInt8 || kind == ProfileKind::kPacked16Bytes;
    const size_t per_warp = bytes ? (size_t)(alphabet + 1) * 32 * rows
                                  : (size_t)(alphabet + 1) * (rows / 4) * 32 * 16;
    return (size_t)kGroupWarps * 3 * kMaxGroups * kRingBytes + tab_bytes(bytes, alphabet) +
           (size_t)kColdWords * 4 * kGroupWarps * 32 + kGroupWarps * per_warp;
}

// The dynamic shared-memory limit of each instantiation is raised once, to
// what the largest alphabet needs, so that concurrent planning of batches
// with different alphabets (from several host threads) never lowers it
// under a launch that needs more.  Occupancy per (profile, alphabet) is
// cached per device.
namespace {
// the ten instantiations, indexed by (profile kind, linear gaps)
using GroupKernel = void (*)(GroupParams);
GroupKernel group_kernel_of(ProfileKind kind, bool lin) {
    switch (kind) {
        case ProfileKind::kInt8:
            return lin ? sw_group_kernel<kRows, true, true, false>
                       : sw_group_kernel<kRows, true, false, false>;
        case ProfileKind::kPacked16:
            return lin ? sw_group_kernel<kRowsPacked, false, true, true>
                       : sw_group_kernel<kRowsPacked, false, false, true>;
        case ProfileKind::kPacked16Bytes:
            return lin ? sw_group_kernel<kRows, true, true, true>
                       : sw_group_kernel<kRows, true, false, true>;
        case ProfileKind::kPacked16R32:
            return lin ? sw_group_kernel<32, false, true, true>
                       : sw_group_kernel<32, false, false, true>;
        default:
            return lin ? sw_group_kernel<kRows, false, true, false>
                       : sw_group_kernel<kRows, false, false, false>;
    }
}
}  // namespace

int group_blocks_per_sm(ProfileKind kind, bool linear, int alphabet, int *smem_bytes) {
    const size_t smem = group_smem_bytes(kind, alphabet);
    if (smem_bytes) *smem_bytes = (int)smem;
    if (alphabet < 1 || alphabet > kMaxAlphabet) return -1;
    constexpr int kMaxDevices = 64;
    static std::mutex mu;
    static int cache[kMaxDevices][2 * kNumProfileKinds][kMaxAlphabet + 1];
    static bool raised[kMaxDevices][2 * kNumProfileKinds];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return -1;
    const int ki = 2 * (int)kind + (linear ? 1 : 0);
    const GroupKernel fn = group_kernel_of(kind, linear);
    std::lock_guard<std::mutex> lk(mu);
    if (cache[dev][ki][alphabet] > 0) return cache[dev][ki][alphabet];
    int optin = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
        cudaSuccess)
        return -1;
    if (smem > (size_t)optin) return 0;  // this alphabet's profile does not fit
    if (!raised[dev][ki]) {
        const int top = (int)std::min<size_t>(group_smem_bytes(kind, kMaxAlphabet), (size_t)optin);
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, top) !=
            cudaSuccess)
            return -1;
        raised[dev][ki] = true;
    }
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fn, kGroupWarps * 32, smem) !=
        cudaSuccess)
        return -1;
    cache[dev][ki][alphabet] = blocks;
    return blocks;
}

cudaError_t launch_group(const GroupParams &p, ProfileKind kind, bool linear, int grid,
                         cudaStream_t s) {
    if (p.n_classes <= 0 || grid <= 0) return cudaSuccess;
    const size_t smem = group_smem_bytes(kind, p.alphabet);
    group_kernel_of(kind, linear)<<<grid, kGroupWarps * 32, smem, s>>>(p);
    return cudaGetLastError();
}

}  // namespace swgb
