// Device helpers shared by the kernels of libae (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ae_internal.h"

#ifndef FULL
#define FULL 0xffffffffu
#endif

namespace aedev {


__device__ __forceinline__ int32_t warp_incl_max(int32_t v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        int32_t o = __shfl_up_sync(FULL, v, d);
        if (lane >= d) v = max(v, o);
    }
    return v;
}

__device__ __forceinline__ uint32_t warp_incl_sum(uint32_t v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t o = __shfl_up_sync(FULL, v, d);
        if (lane >= d) v += o;
    }
    return v;
}

__device__ __forceinline__ int32_t floordiv32(int32_t a, int32_t b) {  // b > 0
    int32_t q = a / b;
    if (q * b != a && a < 0) --q;
    return q;
}

// Theorem 2 threshold of query column j (0-based): an entry lives iff > thr.
// int32 is exact: the engine admits only m * (g + 1) < 2^30, and j <= m.
__device__ __forceinline__ int32_t thr_of(int32_t j, int32_t m, int32_t H, int32_t g) {
    return max(H - 1 - (m - 1 - j) * g, 0);
}

__device__ __forceinline__ int32_t delta_of(const ScoreView &sc, const int8_t *smat, int c, int q) {
    return sc.use_matrix ? (int32_t)smat[c * AE_MAX_SIGMA + q] : (c == q ? sc.sa : sc.sb);
}

// Collections: separator rows among the rows [64 (k / 64), k) of k's block (they
// store letter code 0 but are not occurrences of it; the block's letter counts
// already leave out the separators of earlier blocks), whether row k is one, and
// whether text position p ends a sequence (no alignment crosses it).
__device__ __forceinline__ uint32_t sep_in_block(const IndexView &ix, uint32_t k) {
    const uint32_t *sb = ix.sep + (size_t)(k >> 6) * AE_SEP_BLOCK_WORDS;
    const uint32_t r = k & 63;
    const uint64_t mask = (uint64_t)__ldg(sb + 1) | ((uint64_t)__ldg(sb + 2) << 32);
    return (uint32_t)__popcll(mask & (r ? (~0ull >> (64 - r)) : 0ull));
}
__device__ __forceinline__ bool sep_row(const IndexView &ix, uint32_t k) {
    const uint32_t r = k & 63;
    return ix.sep && ((__ldg(ix.sep + (size_t)(k >> 6) * AE_SEP_BLOCK_WORDS + 1 + (r >> 5)) >> (r & 31)) & 1u);
}
__device__ __forceinline__ bool seq_end(const IndexView &ix, int64_t p) {
    return ix.ends && ((__ldg(ix.ends + (p >> 5)) >> (p & 31)) & 1u);
}

// Occ(c, k): occurrences of letter c in BWT rows [0, k).
__device__ __forceinline__ uint32_t occ_dna(const IndexView &ix, int c, uint32_t k) {
    const uint32_t *blk = ix.occ + (size_t)(k >> 6) * AE_DNA_BLOCK_WORDS;
    const uint4 bits = __ldg(reinterpret_cast<const uint4 *>(blk + 4));
    uint32_t acc = __ldg(blk + c);
    const int r = k & 63;
    const uint32_t w[4] = {bits.x, bits.y, bits.z, bits.w};
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        int take = r - 16 * t;
        take = take < 0 ? 0 : (take > 16 ? 16 : take);
        uint32_t mask = take == 16 ? 0x55555555u : (((1u << (2 * take)) - 1u) & 0x55555555u);
        uint32_t lo = w[t] & 0x55555555u, hi = (w[t] >> 1) & 0x55555555u;
        uint32_t eq = ((c & 1) ? lo : ~lo) & ((c & 2) ? hi : ~hi);
        acc += __popc(eq & mask);
    }
    if (c == 0 && (int64_t)(k >> 6) == (ix.dollar_row >> 6) && (ix.dollar_row & 63) < r) acc -= 1;
    if (c == 0 && ix.sep) acc -= sep_in_block(ix, k);
    return acc;
}

__device__ __forceinline__ uint32_t occ_prot(const IndexView &ix, int c, uint32_t k) {
    const uint32_t *blk = ix.occ + (size_t)(k >> 6) * AE_PROT_BLOCK_WORDS;
    const uint64_t *pl = reinterpret_cast<const uint64_t *>(blk + 22);
    uint32_t acc = __ldg(blk + c);
    const int r = k & 63;
    const uint64_t mask = r ? (~0ull >> (64 - r)) : 0ull;
    uint64_t eq = ~0ull;
#pragma unroll
    for (int t = 0; t < 5; ++t) {
        uint64_t p = __ldg(pl + t);
        eq &= ((c >> t) & 1) ? p : ~p;
    }
    acc += __popcll(eq & mask);
    if (c == 0 && (int64_t)(k >> 6) == (ix.dollar_row >> 6) && (ix.dollar_row & 63) < r) acc -= 1;
    if (c == 0 && ix.sep) acc -= sep_in_block(ix, k);
    return acc;
}

template <int SIGMA>
__device__ __forceinline__ uint32_t occ_of(const IndexView &ix, int c, uint32_t k) {
    return SIGMA == 4 ? occ_dna(ix, c, k) : occ_prot(ix, c, k);
}

// The letter stored in BWT row k (the sentinel row reads as letter 0; callers
// check dollar_row).
template <int SIGMA>
__device__ __forceinline__ int bwt_letter(const IndexView &ix, uint32_t k) {
    const int r = k & 63;
    if (SIGMA == 4) {
        const uint32_t *blk = ix.occ + (size_t)(k >> 6) * AE_DNA_BLOCK_WORDS;
        return (int)((__ldg(blk + 4 + (r >> 4)) >> (2 * (r & 15))) & 3u);
    } else {
        const uint32_t *blk = ix.occ + (size_t)(k >> 6) * AE_PROT_BLOCK_WORDS;
        const uint64_t *pl = reinterpret_cast<const uint64_t *>(blk + 22);
        int code = 0;
#pragma unroll
        for (int t = 0; t < 5; ++t) code |= (int)((__ldg(pl + t) >> r) & 1ull) << t;
        return code;
    }
}

// ---- the int16x2 route of the trie walk.  A row entry's (M, G_a) pair is
// stored in one 32-bit word, M in the low and G_a in the high halfword.  Live
// states are positive and at most depth * g_max, which the engine keeps below
// 32,768 while it uses this route; a dead state is stored as AE_DEAD16, far
// enough from -32,768 that adding a gap charge cannot wrap.
#define AE_DEAD16 (-16000)

__device__ __forceinline__ uint32_t pack_mg(int32_t M, int32_t Ga) {
    const int32_t m = M > 0 ? M : AE_DEAD16, g = Ga > 0 ? Ga : AE_DEAD16;
    return ((uint32_t)m & 0xFFFFu) | ((uint32_t)g << 16);
}
__device__ __forceinline__ int32_t mg_lo(uint32_t v) {
    const int32_t x = (int32_t)(int16_t)(v & 0xFFFFu);
    return x > 0 ? x : AE_NEG;
}
__device__ __forceinline__ int32_t mg_hi(uint32_t v) {
    const int32_t x = (int32_t)(int16_t)(v >> 16);
    return x > 0 ? x : AE_NEG;
}
// Vertical gap of Section 2.2, G_a' = max(G_a + s_s, M + s_g + s_s), on the
// packed pair: swap the halfwords and take one DPX add-max per halfword.
__device__ __forceinline__ int32_t gap_from_mg(uint32_t mg, int32_t ss, int32_t oe) {
    const uint32_t sw = __byte_perm(mg, 0, 0x1032);                       // G_a | M << 16
    const uint32_t c = __vadd2(mg, (uint32_t)oe & 0xFFFFu);                // low: M + s_g + s_s
    const uint32_t r = __viaddmax_s16x2(sw, (uint32_t)ss & 0xFFFFu, c);   // low: max(G_a + s_s, c)
    const int32_t x = (int32_t)(int16_t)(r & 0xFFFFu);
    return x > AE_DEAD16 / 2 ? x : AE_NEG;
}
// The same update on int32 states (AE_NEG stays far below every live value).
__device__ __forceinline__ int32_t gap_from_i32(int32_t M, int32_t Ga, int32_t ss, int32_t oe) {
    return __viaddmax_s32(Ga, ss, M + oe);
}

__device__ __forceinline__ void load_matrix(const ScoreView &sc, int8_t *smat) {
    for (int t = threadIdx.x; t < AE_MAX_SIGMA * AE_MAX_SIGMA; t += blockDim.x) smat[t] = sc.mat[t];
    __syncthreads();
}

// Horizontal-gap finish of one lane's slots (see file comment).  Slot A is at
// column colA with pre-G_b value MpA (already thresholded, AE_NEG if dead);
// optional slot B at colA+1 with MpB.  excl/incl are the exclusive/inclusive
// prefix maxima of the keys M'(k) + k*u over earlier slots (carry included).
// The run covers the columns after the lane's last slot up to next_col - 1,
// where only G_b can be live.
struct SlotOut {
    int32_t MA, MB, GbA, GbB;
    bool aliveA, aliveB;
    int32_t run_start, run_len, run_hits;
};

// The run of columns [run_start, next_col) after a lane's slots, where only
// G_b (key K, the inclusive prefix maximum) can be live: its live cells and
// how many of them reach H.  G_b along the run is v(x) = s_g - x*u + K,
// decreasing; thr(x) is non-decreasing, so the live cells form a prefix.  Most
// runs are empty: the first cell is tested before dividing.  All terms fit
// int32 (the engine checks m * (u + g + 1) < 2^30).
__device__ __forceinline__ void run_of(int32_t run_start, int32_t next_col, int32_t K, const ScoreView &sc,
                                       int32_t m, int32_t H, int32_t u, int32_t &run_len, int32_t &run_hits) {
    run_len = 0;
    run_hits = 0;
    if (K <= AE_KNEG / 2 || run_start >= next_col) return;
    const int32_t g = sc.gmax;
    const int32_t v0 = sc.sg - run_start * u + K;
    if (v0 > thr_of(run_start, m, H, g)) {
        const int32_t x1 = floordiv32(sc.sg + K - 1, u);
        const int32_t x2 = floordiv32(sc.sg + K - H + (m - 1) * g, u + g);
        const int32_t xm = min(min(x1, x2), next_col - 1);
        const int32_t r = xm - run_start + 1;
        if (r > 0) {
            run_len = r;
            if (v0 >= H) {
                const int32_t xh = floordiv32(sc.sg + K - H, u);
                const int32_t rh = min(xh, run_start + r - 1) - run_start + 1;
                run_hits = rh > 0 ? rh : 0;
            }
        }
    }
}

__device__ __forceinline__ void slot_finish(int32_t colA, int32_t MpA, bool hasB, int32_t MpB,
                                            int32_t next_col, int32_t excl, int32_t incl,
                                            const ScoreView &sc, int32_t m, int32_t H, int32_t u,
                                            bool valid, SlotOut &o) {
    const int32_t g = sc.gmax;
    o.GbA = excl > AE_KNEG / 2 ? sc.sg - colA * u + excl : AE_NEG;
    o.MA = max(MpA, o.GbA);
    o.aliveA = valid && o.MA > thr_of(colA, m, H, g);
    o.aliveB = false;
    o.MB = AE_NEG;
    o.GbB = AE_NEG;
    if (valid && hasB) {
        int32_t keyA = MpA > AE_NEG ? MpA + colA * u : AE_KNEG;
        int32_t KB = max(excl, keyA);
        o.GbB = KB > AE_KNEG / 2 ? sc.sg - (colA + 1) * u + KB : AE_NEG;
        o.MB = max(MpB, o.GbB);
        o.aliveB = o.MB > thr_of(colA + 1, m, H, g);
    }
    o.run_start = hasB ? colA + 2 : colA + 1;
    run_of(o.run_start, next_col, valid ? incl : AE_KNEG, sc, m, H, u, o.run_len, o.run_hits);
}

}  // namespace aedev
