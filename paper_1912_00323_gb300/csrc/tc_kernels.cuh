// Tensor-core distance tiles for the high-dimensional path (float input, DP = 8, 16, 32, 64).
//
// The three point phases of the coarse-grid path (the counts of Definition 2, the unions of
// Definitions 3-5 and the labels of Algorithm 4) all test point pairs of neighbouring coarse
// cells against eps.  Here a CTA of 128 threads takes up to 128 rows of one coarse cell (all
// its points for the counts, its core points for the unions, its non-core points for the
// labels) and streams the candidate points of the neighbouring cells (all points for the
// counts, the core points otherwise) in blocks of 128.  Rows and candidates are centred on
// the chunk's first row, c, split into TF32 pairs (hi + lo) and staged in shared memory in the
// K-major, unswizzled operand layout of tcgen05; one thread issues tcgen05.mma kind::tf32
// (K = 8 per instruction, three products per K step: hi.hi + hi.lo + lo.hi) into a 128 x 128
// FP32 accumulator in tensor memory, and every thread reads its row back with tcgen05.ld and
// classifies its 128 pairs.  The rows carry 8 extra K columns (1, 1, 0, ...) and the
// candidates (-hi, -lo, 0, ...) of colA, so the accumulator holds D = x.y - colA directly.
//
// Filter and error bound.  With x = a - c and y = b - c rounded to FP32 and S = |x|^2 + |y|^2,
// d2 = S - 2 x.y is |a - b|^2 up to the centring's rounding (at most 2^-21 S).  The split
// operands represent x and y to 2^-20 relative, the dropped lo.lo product is below 2^-20 of
// |x_i y_i|, every product of TF32 values is exact in FP32, and the accumulation of the
// 3 KP products and the two colA terms adds at most 3 KP 2^-23 of their absolute sum (KP =
// DP + 8 <= 72); with sum |x_i y_i| <= S / 2 and the FP32 norms (2^-18 S) the error of d2 stays
// below 2^-14 S.  With E = 2^-12 S
//   d2 + E < eps^2 (1 - 2^-20)  =>  |a - b|^2 < eps^2 (1 - 2^-22)  (pair within eps),
//   d2 - E > eps^2 (1 + 2^-20)  =>  |a - b|^2 > eps^2 (1 + 2^-21)  (pair outside eps),
// both far enough from eps^2 that the FP64 sum of the exact predicate lands on the same side.
// In terms of D: accept when D > rowA = ((1 + 2^-12) |x|^2 - eps^2 (1 - 2^-20)) / 2 with
// colA = (1 + 2^-12) |y|^2 / 2.  Rejection uses row quantities only: a pair within eps has
// |y|^2 <= 2 |x|^2 + 2 eps^2, so S <= 3 |x|^2 + 2 eps^2 and D >= (|x|^2 - eps^2) / 2 -
// 2^-12 (1.6 |x|^2 + 1.5 eps^2); D < thr_near = (|x|^2 - eps^2) / 2 - 2^-11 (|x|^2 + eps^2)
// (eps^2 taken as eps^2 (1 + 2^-20)) therefore proves the pair outside.  The FP32 rounding
// of these thresholds (a few 2^-24 of S or eps^2) fits in the unused part of the margins,
// because a pair near eps has S >= eps^2 / 2.  Pairs between the two tests are decided by the
// exact predicate on the original coordinates (FP32 filter, FP64 recheck); the counts keep two
// tallies and leave a row that the tallies do not decide to the exact CUDA-core count.  The
// labels are therefore the exact ones.  An
// empty candidate column carries colA = 2^110, so D = -2^110 rejects it.  The host enables these
// kernels only when every extent satisfies d * extent^2 <= 2^100 and eps^2 lies in
// [2^-100, 2^100], so no FP32 value above overflows or loses the bound to underflow.
//
// Residency: each CTA holds 128 of the 512 tensor-memory columns of an SM; the dynamic
// shared memory of these kernels keeps at most four of their CTAs on an SM, so
// tcgen05.alloc never waits for a CTA that is not running.  Every wait on the MMA's mbarrier
// is bounded; a wait that runs out sets the status word, and the CTA stops, waits once more
// (bounded) for the outstanding MMA and frees its tensor memory.
#pragma once

#include "hd_kernels.cuh"

namespace hca {
namespace tc {

constexpr int kTile = 128;                 // rows per chunk (MMA M) and candidates per block (MMA N)
constexpr uint32_t kLBO = 128;             // bytes between core matrices along K
constexpr uint32_t kWaitLimit = 1u << 22;  // mbarrier polls before a wait gives up
constexpr size_t kMinSmem = 48 * 1024;     // per CTA: at most 4 CTAs (4 x 128 TMEM columns) per SM
constexpr int kMaxRng = 32;                // neighbour ranges per cell (the coarse grid has 9)
constexpr uint32_t kSegCand = 16 * kTile;  // unions: candidates per work item (a window of the stream)
constexpr uint32_t kSplitBelow = 32;       // unions: windows only with fewer chunks per CTA than this
enum { kCount = 0, kMerge = 1, kLabels = 2 };

// Unions: core points of neighbour range k of cell A before any pruning (range 0, the cell's
// own pencil, from A on).  The unpruned stream of A is ranges 0 .. n_half - 1 end to end.
__device__ __forceinline__ uint32_t merge_range_len(const uint2 *ranges, int n_all, const uint32_t *cell_start,
                                                    const uint32_t *cx, uint32_t A, int k) {
    uint2 rg = ranges[(uint64_t)A * n_all + k];
    if (k == 0) rg.x = A;
    return rg.x < rg.y ? cx[cell_start[rg.y]] - cx[cell_start[rg.x]] : 0u;
}

// Windows of a 128-row chunk of the unions: one per kSegCand candidates of the unpruned
// stream (an upper bound of the pruned one); window w is the blocks of the pruned stream from
// w * kSegCand on (none when the pruning left fewer).  The items are handed out window-major:
// the first windows of all chunks, then the others, so that no item of a cell with a long
// neighbourhood runs far longer than the rest, and the later windows mostly find the trees that
// the first ones joined (their blocks of one tree are skipped).  With kSplitBelow or more
// chunks per CTA the chunks spread evenly as they are, and each runs whole.
__device__ __forceinline__ uint32_t merge_windows(uint32_t len) {
    return len > kSegCand ? (len + kSegCand - 1u) / kSegCand : 1u;
}

// Cell of work item t: the last c with off[c] <= t, by a 32-way search (one round of loads per
// level instead of one per halving).  A full warp calls it; every lane returns the result.
__device__ __forceinline__ uint32_t chunk_cell_warp(const uint32_t *off, uint32_t C, uint32_t t) {
    const uint32_t lane = threadIdx.x & 31u;
    uint32_t lo = 0, hi = C;  // off[lo] <= t, and off[hi] > t unless hi == C
    while (hi - lo > 1u) {
        const uint32_t step = (hi - lo + 31u) >> 5;
        const uint32_t piv = lo + lane * step;
        const unsigned ok = __ballot_sync(0xffffffffu, piv < hi && __ldg(off + piv) <= t);
        lo += (uint32_t)(31 - __clz(ok)) * step;  // the ok lanes are a prefix (off is nondecreasing)
        hi = min(hi, lo + step);
    }
    return lo;
}

// Row and candidate lists of the three phases.
struct Tables {
    const uint32_t *choff;      // first work item of every coarse cell (this launch)
    const uint32_t *cx;         // exclusive scan of the core flags over sorted points (n + 1)
    const uint32_t *core_list;  // core points, ascending
    const uint32_t *nc_list;    // non-core points, ascending
    const uint32_t *core_lab;   // cluster id of every core point, by core-list index (labels phase)
    const uint32_t *cell_root;  // unions: the one root of a cell's core points (~0 if they differ or
                                // there are none), taken before the phase; nullptr: unused
    const uint32_t *choff_later;  // unions: first item of every coarse cell among the windows after
                                  // the first of its chunks (chunks x (windows - 1) per cell)
    const uint32_t *row_list;     // counts: nullptr = every point of the cell; else the recount of the
                                  // rows the first count handed over (ascending; cx = its scan)
    uint32_t *rc_in, *rc_hi, *rc_done;  // recount, per row of the list: the two tallies summed
                                        // over the windows, and the windows done (zeroed)
};

// A coarse cell whose first tensor-core count handed over at least this many rows counts them
// again on the tensor cores (128 per chunk) instead of leaving them to the CUDA-core count.
// The recount's rows scan their whole neighbourhood (few reach MINPTS early), so each chunk
// runs as windows of kSegCand candidates, one work item each; a row's tallies are summed over
// its windows, and the last window to finish decides the row.
constexpr uint32_t kRecountMin = 32;

// Counts: points of neighbour range k of cell A (the stream is ranges 0 .. n_all - 1 end to end).
__device__ __forceinline__ uint32_t count_range_len(const uint2 *ranges, int n_all, const uint32_t *cell_start,
                                                    uint32_t A, int k) {
    const uint2 rg = ranges[(uint64_t)A * n_all + k];
    return rg.x < rg.y ? cell_start[rg.y] - cell_start[rg.x] : 0u;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Byte offset of element (row, k) in the K-major canonical layout with KP columns: 8 x 16-byte
// core matrices, consecutive along K every kLBO bytes, 8-row groups every KP / 4 core matrices.
template <int KP>
__device__ __forceinline__ uint32_t op_offset(int row, int k) {
    constexpr uint32_t sbo = (KP / 4) * 128;
    return (uint32_t)(row >> 3) * sbo + (uint32_t)(k >> 2) * kLBO + (uint32_t)(row & 7) * 16 + (uint32_t)(k & 3) * 4;
}

// Shared-memory matrix descriptor: start address >> 4, leading and stride byte offsets >> 4,
// descriptor version 1 (bit 46), no swizzle.
template <int KP>
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    constexpr uint32_t sbo = (KP / 4) * 128;
    uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)(kLBO >> 4) << 16;
    d |= (uint64_t)(sbo >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of kind::tf32: D F32 (bit 4), A and B TF32 (bits 7, 10), both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24.
__device__ __forceinline__ uint32_t idesc_tf32() {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTile >> 3) << 17) | ((uint32_t)(kTile >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

// Bounded wait for the completion of the given phase of an mbarrier; false if the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase) {
    uint32_t done = 0;
    for (uint32_t it = 0; it < kWaitLimit && !done; ++it) {
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(mbar), "r"(phase)
            : "memory");
    }
    return done != 0;
}

// 32 consecutive accumulator columns of this warp's 32 lanes (lane i of warp w = row 32 w + i),
// issued without waiting: the registers hold the values after tmem_ld_wait.
__device__ __forceinline__ void tmem_ld32_issue(uint32_t addr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(addr));
}

// Wait for this thread's outstanding tensor-memory loads.  The registers of v pass through the
// wait, so that no use of them is scheduled before it; reg_tie does the same for a second set.
__device__ __forceinline__ void tmem_ld_wait(uint32_t (&v)[32]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]), "+r"(v[7]),
                   "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]), "+r"(v[12]), "+r"(v[13]), "+r"(v[14]), "+r"(v[15]),
                   "+r"(v[16]), "+r"(v[17]), "+r"(v[18]), "+r"(v[19]), "+r"(v[20]), "+r"(v[21]), "+r"(v[22]), "+r"(v[23]),
                   "+r"(v[24]), "+r"(v[25]), "+r"(v[26]), "+r"(v[27]), "+r"(v[28]), "+r"(v[29]), "+r"(v[30]), "+r"(v[31])
                 :
                 : "memory");
}

__device__ __forceinline__ void reg_tie(uint32_t (&v)[32]) {
    asm volatile(""
                 : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]), "+r"(v[7]),
                   "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]), "+r"(v[12]), "+r"(v[13]), "+r"(v[14]), "+r"(v[15]),
                   "+r"(v[16]), "+r"(v[17]), "+r"(v[18]), "+r"(v[19]), "+r"(v[20]), "+r"(v[21]), "+r"(v[22]), "+r"(v[23]),
                   "+r"(v[24]), "+r"(v[25]), "+r"(v[26]), "+r"(v[27]), "+r"(v[28]), "+r"(v[29]), "+r"(v[30]), "+r"(v[31])
                 :
                 : "memory");
}

// Three-input maximum (PTX max.f32 with three sources).
__device__ __forceinline__ float fmax3(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// Largest of 32 FP32 values, as a tree of three-input maxima (17 instructions, four dependent
// steps, instead of a chain of 31).
__device__ __forceinline__ float max32(const uint32_t (&v)[32]) {
    float a[11];
#pragma unroll
    for (int j = 0; j < 10; ++j)
        a[j] = fmax3(__uint_as_float(v[3 * j]), __uint_as_float(v[3 * j + 1]), __uint_as_float(v[3 * j + 2]));
    a[10] = fmaxf(__uint_as_float(v[30]), __uint_as_float(v[31]));
    const float b0 = fmax3(a[0], a[1], a[2]), b1 = fmax3(a[3], a[4], a[5]), b2 = fmax3(a[6], a[7], a[8]);
    const float b3 = fmaxf(a[9], a[10]);
    return fmaxf(fmax3(b0, b1, b2), b3);
}

template <int DP>
struct Smem {
    static constexpr int KP = DP + 8;  // K of the MMA: coordinates and the threshold columns
    float a_hi[kTile * KP];    // rows: centred coordinates (TF32 hi part), (1, 1, 0, ...)
    float a_lo[kTile * KP];    // rows: the lo parts (threshold columns unused)
    float b_hi[kTile * KP];    // candidates: centred coordinates (hi), (-colA_hi, -colA_lo, 0, ...)
    float b_lo[kTile * KP];    // candidates: the lo parts (threshold columns unused)
    float cen[DP];             // the centre c (row 0 of the chunk, original coordinates)
    uint32_t cpay[kTile];      // per candidate: tree node (unions) or cluster id (labels)
    uint32_t cidx[kTile];      // per candidate: list index
    uint32_t gsum[4];          // per 32 candidates: unions: bit mask of the candidates whose tree node
                               // differs from ref; labels: the smallest cluster id
    uint32_t rq0[kMaxRng];     // first list index of each span (a neighbour range, or a kept cell)
    uint32_t rpre[kMaxRng + 1];  // stream offset of each span; [kMaxRng] = stream length
    uint32_t bcell[kMaxRng];   // unions, labels: the neighbour cells, range by range
    uint32_t bnear[kMaxRng];   // 1: some row lies within eps of the cell's box
    uint32_t nbc, bover;       // number of those cells; 1 if they did not fit (no pruning)
    uint32_t cell, nwin;       // the item's coarse cell; unions: windows per chunk of it
    uint32_t la[3], pad3;      // unions: blocks of a look-ahead round not skippable (rotating)
    uint64_t mbar;
    uint32_t taddr, ref, next, pad;
};

template <int DP>
inline size_t smem_bytes() {
    return sizeof(Smem<DP>) > kMinSmem ? sizeof(Smem<DP>) : kMinSmem;
}

// FP32 value truncated to TF32 (10 stored mantissa bits); x - tf32_trunc(x) is exact in FP32.
__device__ __forceinline__ float tf32_trunc(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

// Centre a row (4 coordinates per float4) on c, split it into TF32 hi and lo parts, store both
// in the operand layout (columns [0, DP) of KP) and return the squared norm (FP32) of the
// centred row; an invalid row becomes the zero row.
template <int DP, int KP>
__device__ __forceinline__ float stage_split(float *hi_op, float *lo_op, int row, const float4 (&q)[DP / 4],
                                             const float *c, bool valid) {
    float nrm = 0.f;
#pragma unroll
    for (int k = 0; k < DP / 4; ++k) {
        const float4 cc = *reinterpret_cast<const float4 *>(c + 4 * k);
        float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
        if (valid) {
            w.x = __fsub_rn(q[k].x, cc.x);
            w.y = __fsub_rn(q[k].y, cc.y);
            w.z = __fsub_rn(q[k].z, cc.z);
            w.w = __fsub_rn(q[k].w, cc.w);
        }
        nrm = __fmaf_rn(w.x, w.x, nrm);
        nrm = __fmaf_rn(w.y, w.y, nrm);
        nrm = __fmaf_rn(w.z, w.z, nrm);
        nrm = __fmaf_rn(w.w, w.w, nrm);
        const float4 h = make_float4(tf32_trunc(w.x), tf32_trunc(w.y), tf32_trunc(w.z), tf32_trunc(w.w));
        const float4 l = make_float4(__fsub_rn(w.x, h.x), __fsub_rn(w.y, h.y), __fsub_rn(w.z, h.z), __fsub_rn(w.w, h.w));
        const uint32_t off = op_offset<KP>(row, 4 * k);
        *reinterpret_cast<float4 *>(reinterpret_cast<unsigned char *>(hi_op) + off) = h;
        *reinterpret_cast<float4 *>(reinterpret_cast<unsigned char *>(lo_op) + off) = l;
    }
    return nrm;
}

// Columns [DP, DP + 8) of the hi operand, set once per CTA: the rows' (1, 1, 0, ...) and the
// candidates' trailing zeros (columns DP + 4 .. DP + 7).  The lo operands' threshold columns
// are never read (the threshold K step multiplies the hi parts only).
template <int DP, int KP>
__device__ __forceinline__ void stage_extra_const(float *a_hi, float *b_hi, int row) {
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    const uint32_t o0 = op_offset<KP>(row, DP), o1 = op_offset<KP>(row, DP + 4);
    *reinterpret_cast<float4 *>(reinterpret_cast<unsigned char *>(a_hi) + o0) = make_float4(1.f, 1.f, 0.f, 0.f);
    *reinterpret_cast<float4 *>(reinterpret_cast<unsigned char *>(a_hi) + o1) = z;
    *reinterpret_cast<float4 *>(reinterpret_cast<unsigned char *>(b_hi) + o1) = z;
}

// The candidate's threshold columns: (-colA_hi, -colA_lo, 0, 0) at columns DP .. DP + 3.
template <int DP, int KP>
__device__ __forceinline__ void stage_threshold(float *b_hi, int row, float4 w0) {
    *reinterpret_cast<float4 *>(reinterpret_cast<unsigned char *>(b_hi) + op_offset<KP>(row, DP)) = w0;
}

// box_far for a row held in registers (four coordinates per float4), the box in shared memory.
template <int DP>
__device__ __forceinline__ bool box_far_sh(const float4 (&a)[DP / 4], const float *lo, const float *hi,
                                           const GridParams &g) {
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < DP / 4; ++k) {
        const float4 l = reinterpret_cast<const float4 *>(lo)[k];
        const float4 h = reinterpret_cast<const float4 *>(hi)[k];
        float t = fmaxf(fmaxf(__fsub_rn(l.x, a[k].x), __fsub_rn(a[k].x, h.x)), 0.f); s = __fmaf_rn(t, t, s);
        t = fmaxf(fmaxf(__fsub_rn(l.y, a[k].y), __fsub_rn(a[k].y, h.y)), 0.f);       s = __fmaf_rn(t, t, s);
        t = fmaxf(fmaxf(__fsub_rn(l.z, a[k].z), __fsub_rn(a[k].z, h.z)), 0.f);       s = __fmaf_rn(t, t, s);
        t = fmaxf(fmaxf(__fsub_rn(l.w, a[k].w), __fsub_rn(a[k].w, h.w)), 0.f);       s = __fmaf_rn(t, t, s);
    }
    return s > g.hi32;
}

// The exact predicate on two points of the sorted rows: FP32 filter with the guard band of
// GridParams, FP64 sum in dimension order in the band.
template <int DP>
__device__ __forceinline__ bool within_pts(const float *pts, uint32_t i, uint32_t j, const GridParams &g) {
    const float4 *a = reinterpret_cast<const float4 *>(pts + (uint64_t)i * DP);
    const float4 *b = reinterpret_cast<const float4 *>(pts + (uint64_t)j * DP);
    float av[DP], bv[DP];
#pragma unroll
    for (int k = 0; k < DP / 4; ++k) {
        const float4 x = a[k], y = b[k];
        av[4 * k] = x.x; av[4 * k + 1] = x.y; av[4 * k + 2] = x.z; av[4 * k + 3] = x.w;
        bv[4 * k] = y.x; bv[4 * k + 1] = y.y; bv[4 * k + 2] = y.z; bv[4 * k + 3] = y.w;
    }
    float s = 0.f;
#pragma unroll
    for (int i2 = 0; i2 < DP; ++i2) {
        const float t = __fsub_rn(av[i2], bv[i2]);
        s = __fmaf_rn(t, t, s);
    }
    if (s < g.lo32) return true;
    if (s > g.hi32) return false;
    double e = 0.0;
#pragma unroll
    for (int i2 = 0; i2 < DP; ++i2) {
        const double t = __dsub_rn((double)av[i2], (double)bv[i2]);
        e = __dadd_rn(e, __dmul_rn(t, t));
    }
    return e <= g.eps2;
}

template <int MODE>
__device__ __forceinline__ uint32_t row_point(const Tables &tt, uint32_t k) {
    if (MODE == kCount) return tt.row_list ? __ldg(tt.row_list + k) : k;
    return MODE == kMerge ? __ldg(tt.core_list + k) : __ldg(tt.nc_list + k);
}

// Candidate u of the chunk's stream: the neighbour ranges laid end to end (list indices
// rq0[g] .. rq0[g] + (rpre[g + 1] - rpre[g])).  Returns the list index.
__device__ __forceinline__ uint32_t stream_index(const uint32_t *rpre, const uint32_t *rq0, int n_rng, uint32_t u) {
    int lo = 0, hi = n_rng;  // last g with rpre[g] <= u
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (rpre[mid] <= u) lo = mid; else hi = mid;
    }
    return rq0[lo] + (u - rpre[lo]);
}

// One phase over tensor-core tiles (MODE = kCount, kMerge or kLabels) for the coarse cells
// with at least tc_min[MODE] rows of that phase (the other cells are left to the CUDA-core
// kernels); persistent CTAs take work items from a counter, warp 0 finding the item's cell.
// An item is a 128-row chunk of one cell; for the unions of a call with few chunks, a window
// of kSegCand candidates of a chunk's stream (first windows of all chunks, then the rest).  The
// candidates of an item (its neighbour ranges laid end to end, for the unions and labels only
// the cells whose box some row reaches) stream through in blocks of 128; the next block's rows
// are loaded into registers while the current block is multiplied and classified.
//   kCount:  rows = every point of the cell, candidates = every point of the 27 neighbouring
//            cells; core[p] = (|N_eps(p)| >= MINPTS).  Two tallies per row: pairs surely within
//            eps and pairs not proved outside; a row stops once the first reaches MINPTS.  Once
//            at most tc_handoff rows of a chunk are open the chunk stops, and those rows get
//            core[p] = 2 with their count and the next stream position (or zero and zero for
//            all of them if one saw an undecided pair); a row that ends with MINPTS between
//            the tallies gets core[p] = 2, zero and zero.  The CUDA-core count continues them
//            exactly.  With tt.row_list (the recount): rows = the handed-over rows of the cell,
//            one item per window of kSegCand candidates; the tallies are summed over the
//            windows and the last window of a row decides it the same way.
//   kMerge:  rows = core points, candidates = core points of the upper half of the
//            neighbourhood after the row (each unordered pair once); a pair within eps whose
//            trees differ is joined.  A block whose rows and candidates all share one tree
//            node is skipped before the MMA, and after a skip the next four blocks are tested
//            at once.
//   kLabels: rows = non-core points, candidates = core points of the 27 cells; the row takes
//            the smallest cluster id among the candidates within eps, else -1.
template <int DP, int MODE>
__global__ void __launch_bounds__(kTile) k_tc_hd(HdView<float, DP> v, Tables tt) {
    constexpr int KP = Smem<DP>::KP;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    Smem<DP> &S = *reinterpret_cast<Smem<DP> *>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t mbar = smem_u32(&S.mbar);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.taddr)),
                     "r"(kTile));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    stage_extra_const<DP, KP>(S.a_hi, S.b_hi, tid);  // made visible to the MMA by each block's proxy fence
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t taddr = S.taddr;
    const uint32_t t_lane = taddr + ((uint32_t)(warp * 32) << 16);
    const uint32_t idesc = idesc_tf32();
    const bool recount = MODE == kCount && tt.row_list != nullptr;
    const uint32_t C = v.ctr->n_cells, N0 = recount ? v.ctr->n_tc_recount : v.ctr->n_tc_chunks[MODE];
    uint32_t *const next = recount ? &v.ctr->tc_next_recount : &v.ctr->tc_next[MODE];
    const bool split = MODE == kMerge && N0 < kSplitBelow * gridDim.x;
    const uint32_t NC = split ? N0 + v.ctr->n_tc_chunks[3] : N0;  // unions: first windows, then the rest
    const int n_rng = MODE == kMerge ? v.n_half : v.n_all;
    uint32_t phase = 0;
    bool failed = false;  // CTA-uniform
    uint32_t n_tiles = 0, n_skip = 0, n_re = 0, n_noise = 0;
    unsigned long long n_pairs = 0;  // thread 0: valid rows x valid candidates of the tiles computed

    for (;;) {
        __syncthreads();  // every thread is done with the shared memory of the previous chunk
        if (warp == 0) {  // the next item and its cell (and the unions' windows per chunk)
            uint32_t t = 0;
            if (tid == 0) t = failed ? NC : atomicAdd(next, 1u);
            t = __shfl_sync(0xffffffffu, t, 0);
            uint32_t A = 0, nwin = 1;
            if (t < NC) {
                const bool later = MODE == kMerge && t >= N0;
                A = later ? chunk_cell_warp(tt.choff_later, C, t - N0) : chunk_cell_warp(tt.choff, C, t);
                if (later) {
                    uint32_t len = tid < n_rng ? merge_range_len(v.ranges, v.n_all, v.cell_start, tt.cx, A, tid) : 0u;
                    nwin = merge_windows(__reduce_add_sync(0xffffffffu, len));
                }
                if (recount) {
                    uint32_t len = tid < n_rng ? count_range_len(v.ranges, v.n_all, v.cell_start, A, tid) : 0u;
                    nwin = merge_windows(__reduce_add_sync(0xffffffffu, len));
                }
            }
            if (tid == 0) {
                S.next = t;
                S.cell = A;
                S.nwin = nwin;
            }
        }
        __syncthreads();
        const uint32_t t = S.next;
        if (t >= NC) break;
        const uint32_t A = S.cell;
        const uint32_t aset = set_of_key(v, v.cell_key[A]);
        const GridParams &G = params_of(v, aset);
        const uint32_t cs0 = v.cell_start[A], cs1 = v.cell_start[A + 1];
        uint32_t rbeg, rend;
        if (MODE == kCount) {
            rbeg = tt.row_list ? tt.cx[cs0] : cs0;
            rend = tt.row_list ? tt.cx[cs1] : cs1;
        } else if (MODE == kMerge) {
            rbeg = tt.cx[cs0];
            rend = tt.cx[cs1];
        } else {
            rbeg = cs0 - tt.cx[cs0];
            rend = cs1 - tt.cx[cs1];
        }
        // unions: t < N0: item t - choff[A] = chunk, window 0; then item t - N0 - choff_later[A]
        // = chunk * (nwin - 1) + window - 1
        const bool later = MODE == kMerge && t >= N0;
        const uint32_t item = later ? t - N0 - tt.choff_later[A] : t - tt.choff[A];
        const uint32_t nw = later ? S.nwin - 1u : recount ? S.nwin : 1u;
        const uint32_t win = later ? 1u + item % nw : recount ? item % nw : 0u;
        const uint32_t k0 = rbeg + (uint32_t)kTile * (item / nw);  // list index of row 0
        const uint32_t rk = k0 + (uint32_t)tid;
        const bool have = rk < rend;
        const uint32_t p = have ? row_point<MODE>(tt, rk) : 0u;
        float4 q[DP / 4];
        {
            const float4 *src = reinterpret_cast<const float4 *>(v.pts + (uint64_t)p * DP);
#pragma unroll
            for (int k = 0; k < DP / 4; ++k) q[k] = src[k];  // point 0 past the rows; zeroed when staged
            if (tid == 0) {
#pragma unroll
                for (int k = 0; k < DP / 4; ++k) *reinterpret_cast<float4 *>(S.cen + 4 * k) = q[k];
            }
        }
        // unions and labels: the neighbour cells, then only those whose box lies within eps of
        // some row of the chunk (every thread tests its own row; a cell that no row reaches holds
        // no candidate of this chunk); the stream is one span per kept cell.  Counts keep the
        // whole ranges: the CUDA-core count resumes a handed-over row at a stream position.
        int nspan = n_rng;
        bool by_cell = false;
        if (MODE != kCount) {
            if (warp == 0) {
                uint32_t lo = 0, cnt = 0;
                if (tid < n_rng) {
                    uint2 rg = v.ranges[(uint64_t)A * v.n_all + tid];
                    if (MODE == kMerge && tid == 0) rg.x = A;  // own pencil: this cell and the ones after it
                    if (rg.x < rg.y) {
                        lo = rg.x;
                        cnt = rg.y - rg.x;
                    }
                }
                uint32_t incl = cnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (tid >= o) incl += y;
                }
                const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
                for (uint32_t j = 0; j < cnt; ++j)
                    if (incl - cnt + j < (uint32_t)kMaxRng) S.bcell[incl - cnt + j] = lo + j;
                S.bnear[tid] = 0u;
                if (tid < 3) S.la[tid] = 0u;
                if (tid == 0) {
                    S.nbc = total < (uint32_t)kMaxRng ? total : (uint32_t)kMaxRng;
                    S.bover = total > (uint32_t)kMaxRng ? 1u : 0u;
                }
            }
            __syncthreads();
            by_cell = S.bover == 0u;
            if (by_cell) {
                const uint32_t nbc = S.nbc;
                // the boxes of the listed cells, loaded by all threads at once into b_lo (free
                // until the first block is staged): cell i's lo at 2 DP i, its hi DP further
                float *bx = S.b_lo;
                for (uint32_t f = tid; f < nbc * (DP / 2); f += kTile) {
                    const uint32_t i = f / (DP / 2), r = f % (DP / 2);
                    const uint64_t c = S.bcell[i];
                    const float *src = r < DP / 4 ? v.box_lo + c * DP + 4 * r : v.box_hi + c * DP + 4 * (r - DP / 4);
                    *reinterpret_cast<float4 *>(bx + (size_t)i * 2 * DP + 4 * r) = __ldg(reinterpret_cast<const float4 *>(src));
                }
                __syncthreads();
                if (have)
                    for (uint32_t i = 0; i < nbc; ++i)
                        if (!box_far_sh<DP>(q, bx + (size_t)i * 2 * DP, bx + (size_t)i * 2 * DP + DP, G)) S.bnear[i] = 1u;
                __syncthreads();
                if (warp == 0) {
                    uint32_t q0 = 0, len = 0;
                    bool keep = tid < (int)nbc && S.bnear[tid];
                    if (MODE == kMerge && keep && tt.cell_root) {
                        // two cells whose core points were already all in one tree have no pair
                        // left to join (trees only grow)
                        const uint32_t ra = tt.cell_root[A];
                        keep = ra == 0xffffffffu || tt.cell_root[S.bcell[tid]] != ra;
                    }
                    if (keep) {
                        const uint32_t c = S.bcell[tid];
                        q0 = tt.cx[v.cell_start[c]];
                        const uint32_t q1 = tt.cx[v.cell_start[c + 1]];
                        if (MODE == kMerge && c == A) q0 = max(q0, k0);  // earlier rows pair from their side
                        len = q1 > q0 ? q1 - q0 : 0u;
                    }
                    uint32_t incl = len;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                        if (tid >= o) incl += y;
                    }
                    if (tid < (int)nbc) {
                        S.rq0[tid] = q0;
                        S.rpre[tid] = incl - len;
                    }
                    if (tid == 31) S.rpre[kMaxRng] = incl;  // stream length
                }
                nspan = (int)nbc;
            }
        }
        // the candidate stream: one range per warp-0 lane, then a prefix over the ranges
        if (warp == 0 && !by_cell) {
            uint32_t q0 = 0, len = 0;
            if (tid < n_rng) {
                uint2 rg = v.ranges[(uint64_t)A * v.n_all + tid];
                if (MODE == kMerge && tid == 0) rg.x = A;  // own pencil: this cell and the ones after it
                if (rg.x < rg.y) {
                    q0 = v.cell_start[rg.x];
                    uint32_t q1 = v.cell_start[rg.y];
                    if (MODE != kCount) {
                        q0 = tt.cx[q0];
                        q1 = tt.cx[q1];
                    }
                    if (MODE == kMerge && tid == 0) q0 = max(q0, k0);  // earlier rows pair from their side
                    len = q1 > q0 ? q1 - q0 : 0u;
                }
            }
            uint32_t incl = len;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (tid >= o) incl += y;
            }
            if (tid < n_rng) {
                S.rq0[tid] = q0;
                S.rpre[tid] = incl - len;
            }
            if (tid == 31) S.rpre[kMaxRng] = incl;  // stream length
        }
        __syncthreads();
        // the item's part of the stream: all of it, or for the unions window win of kSegCand
        const uint32_t L_all = S.rpre[kMaxRng];
        const uint32_t u0 = MODE == kMerge || recount ? min(L_all, win * kSegCand) : 0u;
        const uint32_t L = split || recount ? min(L_all, u0 + kSegCand) : L_all;
        if (MODE == kMerge && u0 >= L && win > 0u) continue;  // the pruning left nothing in this window
        const float na = stage_split<DP, KP>(S.a_hi, S.a_lo, tid, q, S.cen, have);
        const float lo = (float)(G.eps2 * (1.0 - 0x1p-20));
        const float hi = (float)(G.eps2 * (1.0 + 0x1p-20));
        const float rowA = 0.5f * __fsub_rn(__fmul_rn(na, 1.000244140625f), lo);  // (1 + 2^-12) |x|^2
        const float thr_near = __fsub_rn(0.5f * __fsub_rn(na, hi), 0x1p-11f * __fadd_rn(na, hi));
        uint32_t cnt = 0, cnt_hi = 0, rp = 0, best = kNoLabel;
        if (MODE == kMerge && have) rp = uf_find(v.parent, p, v.ctr);
        bool done = !have;    // counts: the row surely has MINPTS neighbours
        bool handed = false;  // counts: left to the CUDA-core kernel
        // registers of the next candidate block (loaded one block ahead)
        uint32_t pre_k = 0, pre_pay = 0;
        bool pre_in = false;
        auto prefetch = [&](uint32_t ub) {
            const uint32_t u = ub + (uint32_t)tid;
            pre_in = u < L;
            pre_k = pre_in ? stream_index(S.rpre, S.rq0, nspan, u) : 0u;
            // past the stream: list index 0 (a valid point), zeroed when staged; the loads are
            // not waited for here (no select on their values) but at the staging of the block
            const uint32_t qp = MODE == kCount ? pre_k : __ldg(tt.core_list + pre_k);
            const float4 *src = reinterpret_cast<const float4 *>(v.pts + (uint64_t)qp * DP);
#pragma unroll
            for (int k = 0; k < DP / 4; ++k) q[k] = src[k];
            if (MODE == kMerge) pre_pay = __ldcg(v.parent + qp);  // an ancestor of qp
            if (MODE == kLabels) pre_pay = __ldg(tt.core_lab + pre_k);
        };
        if (u0 < L) prefetch(u0);
        uint32_t la_r = 0;  // unions: look-ahead rounds of this item
        for (uint32_t ub = u0; ub < L; ub += kTile) {
            const bool cin = pre_in;
            const uint32_t nq = min((uint32_t)kTile, L - ub);
            uint32_t rq = 0xffffffffu, ref = 0xffffffffu;
            if (MODE == kMerge) {
                // tree nodes one step further towards the roots; a block whose rows and
                // candidates all share one node is skipped before anything is staged
                if (cin) rq = __ldcg(v.parent + pre_pay);
                if (have) {
                    rp = __ldcg(v.parent + rp);
                    S.ref = rp;  // any row's tree node; all rows write before the barrier
                }
                __syncthreads();
                ref = S.ref;
                if (__syncthreads_and((!have || rp == ref) && (!cin || rq == ref))) {
                    ++n_skip;
                    // look ahead: the tree nodes of the next four blocks' candidates at once
                    // (independent load chains), skipping every block whose candidates all
                    // share the rows' node; the first one that does not is prefetched
                    uint32_t nb = ub + kTile;
                    while (nb < L) {
                        unsigned bad = 0;
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const uint32_t u = nb + (uint32_t)j * kTile + (uint32_t)tid;
                            if (u < L) {
                                const uint32_t k2 = stream_index(S.rpre, S.rq0, nspan, u);
                                const uint32_t x = __ldcg(v.parent + __ldcg(v.parent + __ldg(tt.core_list + k2)));
                                if (x != ref) bad |= 1u << j;
                            }
                        }
                        bad = __reduce_or_sync(0xffffffffu, bad);
                        // slot la_r % 3 was cleared in the previous round (or at the chunk
                        // start); nobody reads slot (la_r + 1) % 3 in this round
                        if ((tid & 31) == 0 && bad) atomicOr(&S.la[la_r % 3u], bad);
                        if (tid == 0) S.la[(la_r + 1u) % 3u] = 0u;
                        __syncthreads();
                        const uint32_t nblk = min(4u, (L - nb + (uint32_t)kTile - 1u) / (uint32_t)kTile);
                        const unsigned stop = S.la[la_r % 3u] | (0xfu << nblk);
                        ++la_r;
                        const uint32_t js = (uint32_t)__ffs(stop) - 1u;  // blocks skipped in this round
                        n_skip += js;
                        nb += js * (uint32_t)kTile;
                        if (js < 4u) break;
                    }
                    if (nb < L) prefetch(nb);
                    ub = nb - (uint32_t)kTile;
                    continue;
                }
                S.cpay[tid] = rq;
                const unsigned dm = __ballot_sync(0xffffffffu, cin && rq != ref);
                if ((tid & 31) == 0) S.gsum[warp] = dm;  // read after the barrier of the MMA wait
            }
            // stage the prefetched block
            {
                const float nb = stage_split<DP, KP>(S.b_hi, S.b_lo, tid, q, S.cen, pre_in);
                const float colA = pre_in ? 0.5f * __fmul_rn(nb, 1.000244140625f) : 0x1p110f;
                const float chi = tf32_trunc(colA);
                stage_threshold<DP, KP>(S.b_hi, tid, make_float4(-chi, -__fsub_rn(colA, chi), 0.f, 0.f));
                S.cidx[tid] = pre_k;
            }
            if (MODE == kLabels) {
                const uint32_t lq = pre_in ? pre_pay : kNoLabel;
                S.cpay[tid] = lq;
                uint32_t gm = lq;
                gm = __reduce_min_sync(0xffffffffu, gm);
                if ((tid & 31) == 0) S.gsum[warp] = gm;
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncthreads();
            asm volatile("tcgen05.fence::after_thread_sync;");
            if (tid == 0) {
                const uint32_t ah = smem_u32(S.a_hi), al = smem_u32(S.a_lo);
                const uint32_t bh = smem_u32(S.b_hi), bl = smem_u32(S.b_lo);
#pragma unroll
                for (int ks = 0; ks < KP / 8; ++ks) {
                    const uint32_t o = ks * 2 * kLBO;
                    mma_tf32(taddr, smem_desc<KP>(ah + o), smem_desc<KP>(bh + o), idesc, ks > 0 ? 1u : 0u);
                    if (ks < DP / 8) {  // the threshold columns have no lo parts
                        mma_tf32(taddr, smem_desc<KP>(ah + o), smem_desc<KP>(bl + o), idesc, 1u);
                        mma_tf32(taddr, smem_desc<KP>(al + o), smem_desc<KP>(bh + o), idesc, 1u);
                    }
                }
                mma_commit(mbar);
            }
            if (ub + kTile < L) prefetch(ub + kTile);  // overlaps the MMA and the classification
            const bool ok = mbar_wait(mbar, phase);
            if (__syncthreads_or(!ok)) {
                failed = true;
                if (tid == 0) set_error(v.ctr, kErrLoop);
                break;
            }
            phase ^= 1u;
            asm volatile("tcgen05.fence::after_thread_sync;");
            ++n_tiles;
            if (tid == 0) n_pairs += (unsigned long long)min((uint32_t)kTile, rend - k0) * nq;
            bool need = have && (MODE != kCount || !done);
            if (__any_sync(0xffffffffu, need)) {
                // counts and labels: 64 columns per wait, the second 32 read even past nq
                // (allocated columns; their values are not used); unions: 32 (the registers
                // of a second set slowed the union-find loop)
                constexpr int NH = MODE == kMerge ? 1 : 2;
                for (uint32_t c0 = 0; c0 < nq; c0 += 32u * NH) {
                    uint32_t dv[NH][32];
                    tmem_ld32_issue(t_lane + c0, dv[0]);
                    if (NH == 2) tmem_ld32_issue(t_lane + c0 + 32, dv[NH - 1]);
                    tmem_ld_wait(dv[0]);
                    if (NH == 2) reg_tie(dv[NH - 1]);
#pragma unroll
                    for (int h = 0; h < NH; ++h) {
                        const uint32_t cg = c0 + 32u * (uint32_t)h;
                        if (cg >= nq || !need) continue;
                        // 32 candidates all proved outside (the common case for the rows that
                        // scan their whole neighbourhood: noise and border points) cost one
                        // maximum each instead of the classification
                        if (MODE == kMerge) {  // the tree's registers push the union loop into spills
                            float mx = __uint_as_float(dv[h][0]);
#pragma unroll
                            for (int j = 1; j < 32; ++j) mx = fmaxf(mx, __uint_as_float(dv[h][j]));
                            if (mx < thr_near) continue;
                        } else if (max32(dv[h]) < thr_near) {
                            continue;
                        }
                        if (MODE == kCount) {
                            // cnt: pairs surely within eps (D > rowA); cnt_hi: pairs not proved
                            // outside (D >= thr_near); four partial tallies each
                            uint32_t ci[4] = {0u, 0u, 0u, 0u}, ch[4] = {0u, 0u, 0u, 0u};
#pragma unroll
                            for (int j = 0; j < 32; ++j) {
                                const float dd = __uint_as_float(dv[h][j]);
                                ci[j & 3] += dd > rowA ? 1u : 0u;
                                ch[j & 3] += dd < thr_near ? 0u : 1u;
                            }
                            cnt += (ci[0] + ci[1]) + (ci[2] + ci[3]);
                            cnt_hi += (ch[0] + ch[1]) + (ch[2] + ch[3]);
                            if (cnt >= G.min_pts) need = false;
                        } else {
                            uint32_t in_m = 0, near_m = 0;
#pragma unroll
                            for (int j = 0; j < 32; ++j) {
                                const float dd = __uint_as_float(dv[h][j]);
                                const bool in = dd > rowA;
                                in_m |= (uint32_t)in << j;
                                near_m |= (uint32_t)(!in && !(dd < thr_near)) << j;
                            }
                            uint32_t m = in_m | near_m;  // near: decided by the exact predicate
                            // candidates sharing the row's tree node need no test; nor do ids
                            // that cannot lower the row's label
                            if (MODE == kMerge && rp == ref) m &= S.gsum[cg >> 5];
                            if (MODE == kLabels && S.gsum[cg >> 5] >= best) m = 0;
                            while (m) {
                                const int j = __ffs(m) - 1;
                                m &= m - 1;
                                const uint32_t col = cg + (uint32_t)j;
                                const bool inside = (in_m >> j) & 1u;
                                const uint32_t ck2 = S.cidx[col];
                                if (MODE == kMerge) {
                                    if (ck2 <= rk || S.cpay[col] == rp) continue;
                                    const uint32_t qp = __ldg(tt.core_list + ck2);
                                    bool hit = inside;
                                    if (!hit) {
                                        ++n_re;
                                        hit = within_pts<DP>(v.pts, p, qp, G);
                                    }
                                    if (hit) {
                                        uf_union(v.parent, p, qp, v.ctr);
                                        rp = uf_find(v.parent, p, v.ctr);
                                        S.cpay[col] = rp;  // now an ancestor of qp too: later rows skip it
                                    }
                                } else {
                                    const uint32_t lq = S.cpay[col];
                                    if (lq >= best) continue;
                                    bool hit = inside;
                                    if (!hit) {
                                        ++n_re;
                                        hit = within_pts<DP>(v.pts, p, __ldg(tt.core_list + ck2), G);
                                    }
                                    if (hit) best = lq;
                                }
                            }
                        }
                    }
                }
            }
            if (MODE == kCount) done = done || cnt >= G.min_pts;
            asm volatile("tcgen05.fence::before_thread_sync;");
            if (MODE == kCount) {
                const int open = __syncthreads_count(!done);
                if (open == 0) break;
                if (!recount && open <= (int)v.tc_handoff && ub + 2 * kTile < L) {
                    // few rows left and more than one block to go: the recount or the CUDA-core
                    // count continues them
                    // the rows resume from the next block if none saw an undecided pair, else
                    // all start over (one start position per chunk)
                    handed = !done;
                    const bool exact = __syncthreads_and(!handed || cnt_hi == cnt) != 0;
                    if (handed) {
                        v.tc_cnt[p] = exact ? cnt : 0u;
                        v.tc_pos[p] = exact ? ub + kTile : 0u;
                    }
                    break;
                }
            } else {
                __syncthreads();
            }
        }
        if (failed) continue;  // the loop head ends this CTA
        if (recount) {
            // this window's tallies (a row that reached MINPTS here stopped early: it is core);
            // the last of the row's windows decides it, as below
            if (have) {
                atomicAdd(tt.rc_in + rk, cnt);
                atomicAdd(tt.rc_hi + rk, cnt_hi);
                __threadfence();
                if (atomicAdd(tt.rc_done + rk, 1u) == nw - 1u) {
                    __threadfence();
                    const uint32_t in = atomicAdd(tt.rc_in + rk, 0u), up = atomicAdd(tt.rc_hi + rk, 0u);
                    const bool is_core = in >= G.min_pts;
                    const bool undecided = !is_core && up >= G.min_pts;
                    if (undecided) {  // counted exactly by the CUDA-core count, from the start
                        v.tc_cnt[p] = 0u;
                        v.tc_pos[p] = 0u;
                    }
                    v.core[p] = undecided ? 2 : (is_core ? 1 : 0);
                    if (is_core) v.cell_core[A] = 1;
                }
            }
        } else if (MODE == kCount) {
            // every candidate seen: a row with cnt < MINPTS <= cnt_hi is counted exactly there
            if (have && !handed && cnt < G.min_pts && cnt_hi >= G.min_pts) {
                handed = true;
                v.tc_cnt[p] = 0u;
                v.tc_pos[p] = 0u;
            }
            const bool is_core = have && !handed && cnt >= G.min_pts;
            if (have) v.core[p] = handed ? 2 : (is_core ? 1 : 0);
            // the unions of a cell may run on the CUDA cores (fewer core rows than points)
            if (__syncthreads_or(is_core) && tid == 0) v.cell_core[A] = 1;
        } else if (MODE == kLabels) {
            if (have) {
                const uint32_t base_label = v.gtab ? (uint32_t)v.set_off[aset] : 0u;
                const int32_t lab = best == kNoLabel ? -1 : (int32_t)(best - base_label);
                const uint32_t o = v.perm[p];
                v.labels[o] = lab;
                if (v.core_out) v.core_out[o] = 0;
                n_noise += lab < 0 ? 1u : 0u;
            }
        }
    }
    if (failed) mbar_wait(mbar, phase);  // the MMA that did not complete in time, bounded again
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(kTile));
    add_counter(&v.ctr->work[6], tid == 0 ? n_tiles : 0u);
    if (tid == 0 && n_pairs) atomicAdd(&v.ctr->tc_pairs, n_pairs);
    add_counter(&v.ctr->work[7], n_re);
    if (MODE == kMerge) add_counter(&v.ctr->work[2], tid == 0 ? n_skip : 0u);
    if (MODE == kLabels) {
        n_noise = __reduce_add_sync(0xffffffffu, n_noise);
        if ((tid & 31) == 0 && n_noise) atomicAdd(&v.ctr->n_noise, n_noise);
    }
}

__device__ __forceinline__ uint32_t tc_chunks(uint32_t rows, uint32_t min_rows) {
    return rows >= min_rows ? (rows + (uint32_t)kTile - 1u) / (uint32_t)kTile : 0u;
}

// The one root of every coarse cell's core points (~0 when they differ or there are none),
// with read-only finds (nothing hooks meanwhile), in three launches so that a cell of
// thousands of points is spread over many warps: clear, one warp per 32-point chunk folding
// its core points' roots into the cell's smallest (lo) and largest (hi) root, then per cell
// lo if lo == hi.
static __global__ void __launch_bounds__(256) k_tc_cell_root_clear(const DevCounters *ctr, uint32_t *__restrict__ lo,
                                                                  uint32_t *__restrict__ hi) {
    const uint32_t C = ctr->n_cells;
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < C; c += gridDim.x * blockDim.x) {
        lo[c] = 0xffffffffu;
        hi[c] = 0u;
    }
}

template <int DP>
__global__ void __launch_bounds__(256) k_tc_cell_root(HdView<float, DP> v, uint32_t *__restrict__ lo,
                                                     uint32_t *__restrict__ hi) {
    const int lane = threadIdx.x & 31;
    const uint32_t C = v.ctr->n_cells, NC = v.ctr->n_chunks;
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < NC; t += warps) {
        const uint32_t A = chunk_cell(v.chunk_off, C, t);
        const uint32_t e = v.cell_start[A + 1], p = v.cell_start[A] + 32u * (t - v.chunk_off[A]) + lane;
        uint32_t mn = 0xffffffffu, mx = 0u;
        if (p < e && v.core[p]) {
            mn = mx = uf_root_readonly(v.parent, p, v.ctr);
        }
        mn = __reduce_min_sync(0xffffffffu, mn);
        mx = __reduce_max_sync(0xffffffffu, mx);
        if (lane == 0 && mn != 0xffffffffu) {
            atomicMin(lo + A, mn);
            atomicMax(hi + A, mx);
        }
    }
}

static __global__ void __launch_bounds__(256) k_tc_cell_root_final(const DevCounters *ctr, uint32_t *__restrict__ lo,
                                                                  const uint32_t *__restrict__ hi) {
    const uint32_t C = ctr->n_cells;
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < C; c += gridDim.x * blockDim.x)
        if (lo[c] != hi[c]) lo[c] = 0xffffffffu;
}

// 128-row chunks of the counts for every coarse cell with at least min_rows points.
static __global__ void __launch_bounds__(256) k_tc_chunks_count(const uint32_t *__restrict__ cell_start,
                                                               const DevCounters *ctr, uint32_t min_rows,
                                                               uint32_t *__restrict__ nch) {
    const uint32_t C = ctr->n_cells;
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < C; c += gridDim.x * blockDim.x)
        nch[c] = tc_chunks(cell_start[c + 1] - cell_start[c], min_rows);
}

// The recount of handed-over rows: their flags (core = 2, set only by the tensor-core count; the
// other cells' flags are still 0), their list (ascending) from the scan hx of the flags, and the
// 128-row chunks of every cell with at least min_rows of them.
static __global__ void __launch_bounds__(256) k_tc_handed_flags(const uint8_t *__restrict__ core, int64_t n,
                                                               uint32_t *__restrict__ f) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        f[j] = core[j] == 2 ? 1u : 0u;
}

static __global__ void __launch_bounds__(256) k_tc_handed_list(const uint8_t *__restrict__ core,
                                                              const uint32_t *__restrict__ hx, int64_t n,
                                                              uint32_t *__restrict__ list) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        if (core[j] == 2) list[hx[j]] = (uint32_t)j;
}

static __global__ void __launch_bounds__(256) k_tc_chunks_recount(const uint32_t *__restrict__ cell_start,
                                                                 const uint32_t *__restrict__ hx,
                                                                 const DevCounters *ctr,
                                                                 const uint2 *__restrict__ ranges, int n_all,
                                                                 uint32_t min_rows, uint32_t *__restrict__ nch) {
    const uint32_t C = ctr->n_cells;
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < C; c += gridDim.x * blockDim.x) {
        uint32_t items = tc_chunks(hx[cell_start[c + 1]] - hx[cell_start[c]], min_rows);
        if (items) {
            uint32_t len = 0;
            for (int k = 0; k < n_all; ++k) len += count_range_len(ranges, n_all, cell_start, c, k);
            items *= merge_windows(len);
        }
        nch[c] = items;
    }
}

// Core flags as uint32 for the scan that numbers the core points.
static __global__ void __launch_bounds__(256) k_tc_core_flags(const uint8_t *__restrict__ core, int64_t n,
                                                             uint32_t *__restrict__ f) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        f[j] = core[j];
}

// Core and non-core point lists (ascending) from the scan cx of the core flags.
static __global__ void __launch_bounds__(256) k_tc_partition(const uint8_t *__restrict__ core,
                                                            const uint32_t *__restrict__ cx, int64_t n,
                                                            uint32_t *__restrict__ core_list,
                                                            uint32_t *__restrict__ nc_list) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t x = cx[j];
        if (core[j]) core_list[x] = (uint32_t)j;
        else nc_list[(uint32_t)j - x] = (uint32_t)j;
    }
}

// Work items of every coarse cell: for the unions, 128-row chunks of core rows (first launch)
// and those chunks times the windows after the first (second launch); for the labels, 128-row
// chunks of non-core rows.
static __global__ void __launch_bounds__(256) k_tc_chunks_split(const uint32_t *__restrict__ cell_start,
                                                               const uint32_t *__restrict__ cx, const DevCounters *ctr,
                                                               const uint2 *__restrict__ ranges, int n_half, int n_all,
                                                               uint32_t min_core, uint32_t min_nc,
                                                               uint32_t *__restrict__ nch_core,
                                                               uint32_t *__restrict__ nch_later,
                                                               uint32_t *__restrict__ nch_nc) {
    const uint32_t C = ctr->n_cells;
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < C; c += gridDim.x * blockDim.x) {
        const uint32_t s = cell_start[c], e = cell_start[c + 1];
        const uint32_t nc = cx[e] - cx[s];
        const uint32_t chunks = tc_chunks(nc, min_core);
        uint32_t later = 0;
        if (chunks) {
            uint32_t len = 0;
            for (int k = 0; k < n_half; ++k) len += merge_range_len(ranges, n_all, cell_start, cx, c, k);
            later = chunks * (merge_windows(len) - 1u);
        }
        nch_core[c] = chunks;
        nch_later[c] = later;
        nch_nc[c] = tc_chunks(e - s - nc, min_nc);
    }
}

// Cluster id of every core point (by core-list index, for the labels phase), its label and
// the core flag output.
template <int DP>
__global__ void __launch_bounds__(256) k_tc_core_labels(HdView<float, DP> v, Tables tt, int nsets,
                                                       uint32_t *__restrict__ core_lab) {
    const uint32_t n_core = tt.cx[v.g.n];
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n_core; k += gridDim.x * blockDim.x) {
        const uint32_t j = tt.core_list[k];
        const uint32_t lab = v.comp_min[v.parent[j]];
        core_lab[k] = lab;
        const uint32_t o = v.perm[j];
        const uint32_t base_label = v.gtab ? (uint32_t)v.set_off[set_of_point(v.set_off, nsets, o)] : 0u;
        v.labels[o] = (int32_t)(lab - base_label);
        if (v.core_out) v.core_out[o] = 1;
    }
}

}  // namespace tc
}  // namespace hca
