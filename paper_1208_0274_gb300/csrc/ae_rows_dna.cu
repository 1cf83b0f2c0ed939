// One trie level of the DNA int16x2 route (Section 5 (3) and Section 2.2),
// organised around the parent entry, in one launch.
//
// A task is a group of up to 32 frontier nodes, one per lane.  Its prologue
// takes each node's child ranges for all four letters from one decode of the
// occurrence block at each end of the node's SA range (Section 5 (3):
// lo' = C[c] + Occ(c, lo), hi' = C[c] + Occ(c, hi)); a single occurrence has
// only the child BWT[lo] (one LF step).  The task then
//
//   counts    per (node, child) the output entries and hits of the child rows,
//   reserves  its ranges in the five output arenas (frontier rows, leaf rows,
//             frontier nodes, leaf injections, range hits) with one atomic
//             per arena on the level's cursors, and
//   writes    the child node records, injections, row entries and range hits:
//             in the walk layout the rows the count phase staged (up to
//             stage_cap entries per lane, DnaRowsArgs) are copied, longer rows
//             and the other layouts are computed a second time.
//
// Rows are computed in one of three layouts chosen per level: short parent
// rows walked one lane per (node, child) in column order (the horizontal gap
// as a running key), long rows spread one parent entry per lane with the
// horizontal gap as a segmented max-plus scan, and levels of few nodes with
// long rows one node per block of WB_T threads (k_rows_dna_wide).  The general
// kernel (ae_trie.cu) handles protein, the int32 route, root rows and cost-tier
// counting; all produce the same nodes and arenas.
#include <cuda_runtime.h>

#include <algorithm>
#include <stdint.h>

#include "ae_device.cuh"
#include "ae_kernels.h"

namespace {
using namespace aedev;

constexpr int DW = 8;   // warps per block
// Resident blocks per SM the kernel is compiled for and launched with (64
// registers a thread)
#ifndef AE_DNA_MINB
#define AE_DNA_MINB 4
#endif

// Occ(c, k) for c = A, C, G, T at once from one 32-byte block (layout in
// ae_internal.h): counts before the block plus the codes of rows [64b, k).
__device__ __forceinline__ void occ4(const IndexView &ix, uint32_t k, uint32_t (&o)[4], uint64_t &w0, uint64_t &w1) {
    const uint32_t *blk = ix.occ + (size_t)(k >> 6) * AE_DNA_BLOCK_WORDS;
    const uint4 cnt = __ldg(reinterpret_cast<const uint4 *>(blk));
    const uint4 bits = __ldg(reinterpret_cast<const uint4 *>(blk + 4));
    w0 = (uint64_t)bits.x | ((uint64_t)bits.y << 32);   // rows 0..31 of the block, 2 bits each
    w1 = (uint64_t)bits.z | ((uint64_t)bits.w << 32);   // rows 32..63
    const uint32_t r = k & 63;
    const uint64_t EV = 0x5555555555555555ull;
    const uint64_t m0 = r >= 32 ? EV : (((1ull << (2 * r)) - 1) & EV);
    const uint64_t m1 = r <= 32 ? 0ull : (((1ull << (2 * (r - 32))) - 1) & EV);
    const uint64_t l0 = w0 & EV, h0 = (w0 >> 1) & EV, l1 = w1 & EV, h1 = (w1 >> 1) & EV;
    const uint32_t nC = __popcll(l0 & ~h0 & m0) + __popcll(l1 & ~h1 & m1);
    const uint32_t nG = __popcll(~l0 & h0 & m0) + __popcll(~l1 & h1 & m1);
    const uint32_t nT = __popcll(l0 & h0 & m0) + __popcll(l1 & h1 & m1);
    uint32_t nA = r - nC - nG - nT;
    if ((int64_t)(k >> 6) == (ix.dollar_row >> 6) && (uint32_t)(ix.dollar_row & 63) < r) nA -= 1;
    if (ix.sep) nA -= sep_in_block(ix, k);   // collections: separator rows store code 0
    o[0] = cnt.x + nA;
    o[1] = cnt.y + nC;
    o[2] = cnt.z + nG;
    o[3] = cnt.w + nT;
}

// Child ranges of SA range [lo, hi) for the four letters; returns the mask of
// non-empty children.
__device__ __forceinline__ unsigned kids4(const IndexView &ix, uint32_t lo, uint32_t hi, uint32_t (&clo)[4],
                                          uint32_t (&chi)[4]) {
    uint32_t a[4], b[4];
    uint64_t w0, w1;
    occ4(ix, lo, a, w0, w1);
    if (hi - lo == 1) {
        if ((int64_t)lo == ix.dollar_row || sep_row(ix, lo)) return 0u;
        const uint32_t r = lo & 63;
        const int c = (int)(((r < 32 ? w0 : w1) >> (2 * (r & 31))) & 3ull);
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            clo[x] = ix.C[x] + a[x];
            chi[x] = clo[x] + (x == c ? 1u : 0u);
        }
        return 1u << c;
    }
    occ4(ix, hi, b, w0, w1);
    unsigned mask = 0;
#pragma unroll
    for (int x = 0; x < 4; ++x) {
        clo[x] = ix.C[x] + a[x];
        chi[x] = ix.C[x] + b[x];
        if (chi[x] > clo[x]) mask |= 1u << x;
    }
    return mask;
}

// Per-warp shared state of a task, per (node lane, letter): the outputs and
// hits counted so far (count phase) or the next output positions relative to
// the task's arena bases (write phase), the counted totals (the write phase's
// bounds) and the child's SA range.
struct WarpSmem {
    uint32_t a[128];    // count: entries   write: next entry position
    uint32_t h[128];    // count: hits      write: next hit position
    uint32_t be[128];   // write: the child's counted entries
    uint32_t bh[128];   // write: the child's counted hits
    uint32_t lo[128];   // child SA range
    uint32_t hi[128];
    uint32_t sinfo[128];   // walk layout: a staged child row: 1 << 31 | lane << 16 | first entry; 0: not staged
    int32_t carry[4];   // per child index: the G_b scan's carry into the next chunk
    uint64_t base[3];   // write: the task's first slot in the frontier, leaf and hit arenas
};

// Length of a gap run (Section 2.2: a horizontal gap extended column by column)
// without a division: the run after a lane's last slot starts at column rs with
// G_b = V0 > 0 and loses u per column, so away from the query's last columns
// (threshold 0) its live cells number floor((V0 - 1) / u) + 1.  The quotient is
// taken as a product with the reciprocal rec = ceil(2^32 / u), exact for
// numerators below 2^16 (the int16x2 route keeps every state below 2^15).
__device__ __forceinline__ uint32_t div_small(uint32_t a, uint64_t rec) {
    return (uint32_t)(((uint64_t)a * rec) >> 32);
}

__device__ __forceinline__ uint64_t reduce_add_u64(uint32_t v) {
    const uint32_t hi = __reduce_add_sync(FULL, v >> 16), lo = __reduce_add_sync(FULL, v & 0xFFFFu);
    return ((uint64_t)hi << 16) + lo;
}

__device__ __forceinline__ uint32_t excl_scan_u32(uint32_t v) {
    const int lane = threadIdx.x & 31;
    uint32_t x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, x, d);
        if (lane >= d) x += y;
    }
    return x - v;
}

__device__ __forceinline__ uint64_t excl_scan_u64(uint64_t v, uint64_t &total) {
    const int lane = threadIdx.x & 31;
    uint64_t x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint64_t y = __shfl_up_sync(FULL, x, d);
        if (lane >= d) x += y;
    }
    total = __shfl_sync(FULL, x, 31);
    return x - v;
}

// Rows of short parent rows, one lane per (node, child): the lane walks the
// parent row entry by entry in column order and carries the horizontal gap as
// a running key (the recurrence of Section 2.2 in its sequential form), so no
// scan, vote or compaction is needed; siblings sit in adjacent lanes and read
// the same parent entries.  Count phase: the pair's entries and hits go to its
// (node, letter) slot.  Write phase: the pair writes its child row from the
// slot's position on.  The values equal those of the lane-per-entry form.
template <bool WRITE>
__device__ __forceinline__ void rows_seq(const DnaRowsArgs &a, WarpSmem &sm, int lane, unsigned kmask, unsigned smask,
                                         uint32_t len, uint64_t noff, int32_t qm, int32_t qH, int32_t tbase,
                                         uint32_t qoff, int32_t qid) {
    const ScoreView &sc = a.sc;
    const int32_t u = -sc.ss, oe = sc.sg + sc.ss, g = sc.gmax, sa = sc.sa, sb = sc.sb;
    const int32_t strong = -oe;
    // pairs are handed out in rounds of 32 in order of decreasing row length (a
    // bitonic sort of the node lanes by length), so that the lanes of a round walk
    // rows of similar length
    uint32_t key = (kmask ? min(len, (1u << 26) - 1u) : 0u) << 5 | (uint32_t)(31 - lane);   // distinct per lane
    // with at most 32 pairs there is a single round, whose length no order changes
    if (__reduce_add_sync(FULL, (uint32_t)__popc(kmask)) > 32) {
#pragma unroll
        for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
            for (int jj = k >> 1; jj > 0; jj >>= 1) {
                const uint32_t other = __shfl_xor_sync(FULL, key, jj);
                const bool up = ((lane & k) == 0);          // this block sorts descending
                const bool low = (lane & jj) == 0;
                key = (low == up) ? max(key, other) : min(key, other);
            }
        }
    }
    const int sorted_lane = 31 - (int)(key & 31u);      // the node lane at this sorted position
    const uint32_t np = __popc(__shfl_sync(FULL, kmask, sorted_lane));   // its pairs
    uint32_t poff = np;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, poff, d);
        if (lane >= d) poff += y;
    }
    const uint32_t npairs = __shfl_sync(FULL, poff, 31);
    poff -= np;
    // count phase: this lane's staging region (its pairs' rows one after another)
    uint2 *stg = nullptr;
    if (!WRITE && a.stage)
        stg = a.stage + ((int64_t)(blockIdx.x * DW + (threadIdx.x >> 5)) * 32 + lane) * a.stage_cap;
    uint32_t sf = 0;   // entries staged so far in this task
    for (uint32_t p0 = 0; p0 < npairs; p0 += 32) {
        const uint32_t p = p0 + lane;
        const bool valid = p < npairs;
        int S = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const uint32_t o = __shfl_sync(FULL, poff, S + step);
            if (o <= p) S += step;
        }
        const uint32_t i = p - __shfl_sync(FULL, poff, S);
        const int L = __shfl_sync(FULL, sorted_lane, S);
        unsigned km = __shfl_sync(FULL, kmask, L);
        const unsigned smL = __shfl_sync(FULL, smask, L);
        const uint32_t nlen = __shfl_sync(FULL, len, L);
        const uint64_t off = __shfl_sync(FULL, noff, L);
        const int32_t m = __shfl_sync(FULL, qm, L), H = __shfl_sync(FULL, qH, L);
        const int32_t tb0 = __shfl_sync(FULL, tbase, L);
        const uint32_t qo = __shfl_sync(FULL, qoff, L);
        const int32_t eq = __shfl_sync(FULL, qid, L);
        if (!valid) continue;
        for (uint32_t x = 0; x < i; ++x) km &= km - 1;   // the i-th child letter of the node
        const int c = __ffs(km) - 1;
        const bool st = (smL >> c) & 1u;
        const int slot = L * 4 + c;
        const uint8_t *P = a.qv.codes + qo;
        uint64_t eout = 0, hout = 0;
        uint32_t clo = 0, chi = 0, ebud = 0, hbud = 0;   // write phase: the child's outputs as counted
        if (WRITE) {
            eout = sm.base[st ? 0 : 1] + sm.a[slot];
            hout = sm.base[2] + sm.h[slot];
            clo = sm.lo[slot];
            chi = sm.hi[slot];
            ebud = sm.be[slot];
            hbud = sm.bh[slot];
        }
        uint32_t cnt = 0, hcnt = 0;
        bool bad = false;
        const uint32_t sf0 = sf;   // count phase: where this pair's row starts in the staging region
        int32_t K = AE_KNEG, prev_j = -2, prev_M = 0;
        const int32_t *pjr = a.pj + off;     // the parent row
        const uint32_t *pmr = a.pmg + off;
        // loads run ahead of their use: the next entry and its query letters, and
        // the column of the entry after it
        int32_t j_c = pjr[0];
        uint32_t mg_c = pmr[0];
        int32_t j_n = nlen > 1 ? pjr[1] : m;
        // a parent row is sorted by column inside [0, m): its first column is checked
        // here and every next one against the previous and m below; anything else is
        // reported, and no column past the query is read
        if ((uint32_t)j_c >= (uint32_t)m) bad = true;
        int pa_c = !bad ? (int)P[j_c] : 255;
        int pb_c = !bad && j_c + 1 < m ? (int)P[j_c + 1] : 255;
        for (uint32_t k = 0; k < nlen && !bad; ++k) {
            const int32_t j = j_c, jn = j_n;
            const uint32_t mg = mg_c;
            const int pA = pa_c, pB = pb_c;
            if (jn <= j || jn > m) {
                bad = true;
                break;
            }
            if (k + 1 < nlen) {
                mg_c = pmr[k + 1];
                j_c = jn;
                j_n = (k + 2 < nlen) ? pjr[k + 2] : m;
                // a next column at m is reported in its own step (no later column is above it)
                pa_c = jn < m ? (int)P[jn] : 255;
                pb_c = jn + 1 < m ? (int)P[jn + 1] : 255;
            }
            const int32_t M = (int32_t)(int16_t)(mg & 0xFFFFu);
            const int32_t traw = tb0 + j * g;
            const int32_t tA = max(traw, 0), tB = max(traw + g, 0);
            const int32_t ju = j * u;
            // the vertical gap, max(G_a + s_s, M + s_g + s_s); a dead state (stored as
            // AE_DEAD16) stays far below the threshold, which is >= 0
            int32_t Gap = max((int32_t)(int16_t)(mg >> 16) + sc.ss, M + oe);
            Gap = Gap > tA ? Gap : AE_NEG;
            int32_t DA = (prev_j + 1 == j && prev_M > 0) ? prev_M + (c == pA ? sa : sb) : AE_NEG;
            DA = DA > tA ? DA : AE_NEG;
            const int32_t MpA = max(DA, Gap);
            const int32_t MA = max(MpA, K > AE_KNEG / 2 ? sc.sg - ju + K : AE_NEG);
            const bool aliveA = MA > tA;
            if (MpA > strong) K = max(K, MpA + ju);
            const bool hasB = (j + 1 < m) && (j + 1 != jn);
            int32_t MB = AE_NEG;
            bool aliveB = false;
            if (hasB) {
                const int32_t DB = M + (c == pB ? sa : sb);
                const int32_t MpB = DB > tB ? DB : AE_NEG;
                MB = max(MpB, K > AE_KNEG / 2 ? sc.sg - ju - u + K : AE_NEG);
                aliveB = MB > tB;
                if (MpB > strong) K = max(K, MpB + ju + u);
            }
            // the gap run after the slots: columns [rs, jn) where only G_b lives
            int32_t run_len = 0, run_hits = 0;
            const int32_t rs = hasB ? j + 2 : j + 1;
            const int32_t V0 = sc.sg - rs * u + K;
            if (K > AE_KNEG / 2 && rs < jn && V0 > 0) {
                const int32_t rl = min((int32_t)div_small((uint32_t)(V0 - 1), a.urec) + 1, jn - rs);
                if (traw + (rs + rl - 1) * g <= 0) {
                    run_len = rl;
                    if (V0 >= H) run_hits = min(rl, (int32_t)div_small((uint32_t)(V0 - H), a.urec) + 1);
                } else {
                    run_of(rs, jn, K, sc, m, H, u, run_len, run_hits);
                }
            }
            const bool hA = st && aliveA && MA >= H, hB = st && aliveB && MB >= H;
            if (!WRITE) {
                const uint32_t n = (uint32_t)aliveA + (uint32_t)aliveB + (uint32_t)run_len;
                cnt += n;
                hcnt += (uint32_t)hA + (uint32_t)hB + (st ? (uint32_t)run_hits : 0u);
                if (stg && n) {
                    if (sf + n > (uint32_t)a.stage_cap) {
                        stg = nullptr;   // the region is full: this and the later pairs are computed again
                    } else {
                        if (aliveA) stg[sf++] = make_uint2((uint32_t)j, pack_mg(MA, Gap));
                        if (aliveB) stg[sf++] = make_uint2((uint32_t)(j + 1), pack_mg(MB, AE_NEG));
                        for (int32_t r = 0; r < run_len; ++r)
                            stg[sf++] = make_uint2((uint32_t)(rs + r), pack_mg(V0 - r * u, AE_NEG));
                    }
                }
            } else if (!bad) {
                // every write stays inside the child's own range, as the count phase sized it
                if (cnt + (uint32_t)aliveA + (uint32_t)aliveB + (uint32_t)run_len > ebud ||
                    hcnt + (uint32_t)hA + (uint32_t)hB + (st ? (uint32_t)run_hits : 0u) > hbud) {
                    bad = true;   // the phases disagree: reported, not written
                } else {
                    if (aliveA) {
                        if (st) {
                            a.fj[eout + cnt] = j;
                            a.fmg[eout + cnt] = pack_mg(MA, Gap);
                        } else {
                            a.lj[eout + cnt] = j;
                            a.lM[eout + cnt] = MA;
                            a.lGa[eout + cnt] = Gap;
                        }
                        ++cnt;
                        if (hA) a.rhits[hout + hcnt++] = RangeHit{clo, chi, eq, j, MA, 0};
                    }
                    if (aliveB) {
                        if (st) {
                            a.fj[eout + cnt] = j + 1;
                            a.fmg[eout + cnt] = pack_mg(MB, AE_NEG);
                        } else {
                            a.lj[eout + cnt] = j + 1;
                            a.lM[eout + cnt] = MB;
                            a.lGa[eout + cnt] = AE_NEG;
                        }
                        ++cnt;
                        if (hB) a.rhits[hout + hcnt++] = RangeHit{clo, chi, eq, j + 1, MB, 0};
                    }
                    for (int32_t r = 0; r < run_len; ++r) {
                        const int32_t col = rs + r, val = V0 - r * u;
                        if (st) {
                            a.fj[eout + cnt] = col;
                            a.fmg[eout + cnt] = pack_mg(val, AE_NEG);
                        } else {
                            a.lj[eout + cnt] = col;
                            a.lM[eout + cnt] = val;
                            a.lGa[eout + cnt] = AE_NEG;
                        }
                        ++cnt;
                        if (st && r < run_hits) a.rhits[hout + hcnt++] = RangeHit{clo, chi, eq, col, val, 0};
                    }
                }
            }
            prev_j = j;
            prev_M = M;
        }
        if (!WRITE) {
            sm.a[slot] = cnt;
            sm.h[slot] = hcnt;
            sm.sinfo[slot] = (stg && !bad) ? (0x80000000u | ((uint32_t)lane << 16) | sf0) : 0u;
        }
        if (bad) atomicExch(&a.ctr->overflow, 1ull);
    }
}

// Rows of long parent rows: the task's parent entries laid end to end over the
// lanes, 32 at a time, one entry per lane; each lane computes the slots of its
// entry for every child of its node (G_a once, the diagonal terms per child)
// and the horizontal gaps are a max-plus scan segmented by node.  `woff` is
// the lane's node's first entry in the task, `total` the task's entries.
template <bool WRITE>
__device__ __forceinline__ void rows_spread(const DnaRowsArgs &a, WarpSmem &sm, int lane, unsigned kmask,
                                            unsigned smask, uint32_t len, uint64_t noff, int32_t qm, int32_t qH,
                                            int32_t tbase, uint32_t qoff, int32_t qid, uint32_t woff,
                                            uint32_t total) {
    const ScoreView &sc = a.sc;
    const int32_t u = -sc.ss, oe = sc.sg + sc.ss, g = sc.gmax, sa = sc.sa, sb = sc.sb;
    const int32_t strong = -oe;   // a gap state from M' can be live only if M' > |s_g + s_s| (Eq. 3)
    const unsigned le = (lane == 31) ? 0xffffffffu : ((1u << (lane + 1)) - 1u);
    // ---- the rows: parent entries laid end to end over the lanes
    if (lane < 4) sm.carry[lane] = AE_KNEG;
    __syncwarp();
    for (uint32_t t0 = 0; t0 < total; t0 += 32) {
        const uint32_t t = t0 + lane;
        const bool valid = t < total;
        int L = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const uint32_t o = __shfl_sync(FULL, woff, L + step);
            if (o <= t) L += step;
        }
        const uint32_t k = t - __shfl_sync(FULL, woff, L);
        const uint32_t nlen = __shfl_sync(FULL, len, L);
        const uint64_t off = __shfl_sync(FULL, noff, L);
        const unsigned km = __shfl_sync(FULL, kmask, L);
        const unsigned sm_ = __shfl_sync(FULL, smask, L);
        const int32_t m = __shfl_sync(FULL, qm, L);
        const int32_t H = __shfl_sync(FULL, qH, L);
        const int32_t tb0 = __shfl_sync(FULL, tbase, L);
        const uint32_t qo = __shfl_sync(FULL, qoff, L);
        const int32_t eq = WRITE ? __shfl_sync(FULL, qid, L) : 0;   // query of the entry's node
        const unsigned heads = __ballot_sync(FULL, !valid || k == 0 || lane == 0);
        const int first_lane = 31 - __clz(heads & le);
        const bool next_in = (lane < 31) && (((heads >> (lane + 1)) & 1u) == 0);
        const bool is_last = valid && !next_in;
        int32_t j = m;
        uint32_t mg = 0;
        if (valid) {
            j = a.pj[off + k];
            mg = a.pmg[off + k];
        }
        const int32_t M = (int32_t)(int16_t)(mg & 0xFFFFu);   // live iff > 0
        int32_t jn = __shfl_down_sync(FULL, j, 1);
        int32_t pjv = __shfl_up_sync(FULL, j, 1), pMv = __shfl_up_sync(FULL, M, 1);
        if (valid) {
            if (!next_in) jn = (k + 1 < nlen) ? a.pj[off + k + 1] : m;
            if (lane == first_lane) {
                if (k > 0) {
                    pjv = a.pj[off + k - 1];
                    pMv = (int32_t)(int16_t)(a.pmg[off + k - 1] & 0xFFFFu);
                } else {
                    pjv = -2;
                    pMv = 0;
                }
            }
        }
        const uint8_t *P = a.qv.codes + qo;
        const bool adjA = valid && pjv + 1 == j && pMv > 0;
        const bool hasB = valid && (j + 1 < m) && (j + 1 != jn);
        const int pA = (valid && (uint32_t)j < (uint32_t)m) ? (int)P[j] : 255;   // never past the query
        const int pB = hasB ? (int)P[j + 1] : 255;
        const int32_t traw = tb0 + j * g;
        const int32_t tA = max(traw, 0), tB = max(traw + g, 0);
        int32_t Gap = valid ? max((int32_t)(int16_t)(mg >> 16) + sc.ss, M + oe) : AE_NEG;   // dead stays below tA >= 0
        Gap = Gap > tA ? Gap : AE_NEG;
        const int32_t ju = j * u;
        // the node continuing from the previous chunk sits at lane 0
        const uint32_t k_lane0 = __shfl_sync(FULL, k, 0);
        const bool cont = first_lane == 0 && valid && k_lane0 > 0;
        const bool goes_on = __shfl_sync(FULL, (int)(valid && k + 1 < nlen), 31) != 0;
        unsigned rem = valid ? km : 0u;
#pragma unroll 1
        for (int i = 0; i < 4; ++i) {
            const bool has_c = rem != 0;
            if (!__any_sync(FULL, has_c)) {
                if (lane == 0) sm.carry[i] = AE_KNEG;
                __syncwarp();
                continue;
            }
            const int c = has_c ? __ffs(rem) - 1 : 0;
            rem &= rem - 1;
            int32_t MpA = AE_NEG, MpB = AE_NEG;
            if (has_c) {
                int32_t DA = adjA ? pMv + (c == pA ? sa : sb) : AE_NEG;
                DA = DA > tA ? DA : AE_NEG;
                MpA = max(DA, Gap);
                int32_t DB = M + (c == pB ? sa : sb);
                MpB = (hasB && DB > tB) ? DB : AE_NEG;
            }
            const int32_t keyA = MpA > strong ? MpA + ju : AE_KNEG;
            const int32_t keyB = MpB > strong ? MpB + ju + u : AE_KNEG;
            int32_t incl = max(keyA, keyB);
            int32_t excl = AE_KNEG;
            const int32_t cin = sm.carry[i];
            if (__any_sync(FULL, incl > AE_KNEG || (cont && cin > AE_KNEG))) {
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const int32_t o = __shfl_up_sync(FULL, incl, d);
                    if (lane - d >= first_lane) incl = max(incl, o);
                }
                if (cont) incl = max(incl, cin);
                excl = __shfl_up_sync(FULL, incl, 1);
                if (lane - 1 < first_lane) excl = cont ? cin : AE_KNEG;
            }
            __syncwarp();
            if (lane == 31) sm.carry[i] = goes_on ? incl : AE_KNEG;
            // finish: G_b at the slots, then the gap run after them
            const int32_t GbA = excl > AE_KNEG / 2 ? sc.sg - ju + excl : AE_NEG;
            const int32_t MA = max(MpA, GbA);
            const bool aliveA = has_c && MA > tA;
            int32_t MB = AE_NEG;
            bool aliveB = false;
            if (has_c && hasB) {
                const int32_t KB = max(excl, keyA);
                const int32_t GbB = KB > AE_KNEG / 2 ? sc.sg - ju - u + KB : AE_NEG;
                MB = max(MpB, GbB);
                aliveB = MB > tB;
            }
            // the gap run after the lane's slots: columns [run_start, jn) where only G_b
            // can live, G_b(x) = V0 - (x - run_start) u
            int32_t run_len = 0, run_hits = 0;
            const int32_t run_start = hasB ? j + 2 : j + 1;
            const int32_t V0 = sc.sg - run_start * u + incl;
            if (has_c && incl > AE_KNEG / 2 && run_start < jn && V0 > 0) {
                const int32_t rl = min((int32_t)div_small((uint32_t)(V0 - 1), a.urec) + 1, jn - run_start);
                if (traw + (run_start + rl - 1) * g <= 0) {   // threshold 0 over the whole run
                    run_len = rl;
                    if (V0 >= H) run_hits = min(rl, (int32_t)div_small((uint32_t)(V0 - H), a.urec) + 1);
                } else {                                       // the query's last columns: exact form
                    run_of(run_start, jn, incl, sc, m, H, u, run_len, run_hits);
                }
            }
            const bool st = has_c && ((sm_ >> c) & 1u);
            const bool hA = st && aliveA && MA >= H, hB = st && aliveB && MB >= H;
            const uint32_t cnt = (uint32_t)aliveA + (uint32_t)aliveB + (uint32_t)run_len;
            const uint32_t hcnt = (uint32_t)hA + (uint32_t)hB + (st ? (uint32_t)run_hits : 0u);
            const unsigned in_seg = le & ~((1u << first_lane) - 1u);
            uint32_t ci, hi;
            if (__any_sync(FULL, run_len > 0)) {
                ci = cnt;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const uint32_t x = __shfl_up_sync(FULL, ci, d);
                    if (lane - d >= first_lane) ci += x;
                }
            } else {
                ci = __popc(__ballot_sync(FULL, aliveA) & in_seg) + __popc(__ballot_sync(FULL, aliveB) & in_seg);
            }
            if (__any_sync(FULL, run_hits > 0)) {
                hi = hcnt;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const uint32_t y = __shfl_up_sync(FULL, hi, d);
                    if (lane - d >= first_lane) hi += y;
                }
            } else {
                hi = __popc(__ballot_sync(FULL, hA) & in_seg) + __popc(__ballot_sync(FULL, hB) & in_seg);
            }
            const int slot = L * 4 + c;
            if (!WRITE) {
                if (is_last && has_c) {
                    sm.a[slot] += ci;
                    sm.h[slot] += hi;
                }
                __syncwarp();
                continue;
            }
            // ---- write the entries (and the hits of children that stay)
            uint64_t e0 = 0, h0 = 0;
            if (has_c) {
                e0 = sm.base[st ? 0 : 1] + sm.a[slot] + (ci - cnt);
                h0 = sm.base[2] + sm.h[slot] + (hi - hcnt);
            }
            __syncwarp();
            if (is_last && has_c) {
                sm.a[slot] += ci;
                sm.h[slot] += hi;
            }
            // the outputs stay inside their arenas even if the two phases ever
            // disagreed: such a chunk is reported (overflow) and not written
            const bool outside = has_c && (e0 + cnt > (st ? a.fr_ent_cap : a.lf_ent_cap) ||
                                           h0 + hcnt > a.hit_cap);
            if (__any_sync(FULL, outside)) {
                if (lane == 0) atomicExch(&a.ctr->overflow, 1ull);
                __syncwarp();
                continue;
            }
            if (aliveA) {
                if (st) {
                    a.fj[e0] = j;
                    a.fmg[e0] = pack_mg(MA, Gap);
                } else {
                    a.lj[e0] = j;
                    a.lM[e0] = MA;
                    a.lGa[e0] = Gap;
                }
            }
            if (aliveB) {
                const uint64_t eb = e0 + (aliveA ? 1 : 0);
                if (st) {
                    a.fj[eb] = j + 1;
                    a.fmg[eb] = pack_mg(MB, AE_NEG);
                } else {
                    a.lj[eb] = j + 1;
                    a.lM[eb] = MB;
                    a.lGa[eb] = AE_NEG;
                }
            }
            if (hA || hB) {
                const RangeHit base_hit = {sm.lo[slot], sm.hi[slot], eq, 0, 0, 0};
                uint64_t hp = h0;
                if (hA) {
                    RangeHit r = base_hit;
                    r.j = j;
                    r.score = MA;
                    a.rhits[hp++] = r;
                }
                if (hB) {
                    RangeHit r = base_hit;
                    r.j = j + 1;
                    r.score = MB;
                    a.rhits[hp] = r;
                }
            }
            if (run_len > 0) {   // each lane writes its own run (a few cells)
                const uint64_t er = e0 + (uint64_t)aliveA + (uint64_t)aliveB;
                const uint64_t hr = h0 + (uint64_t)hA + (uint64_t)hB;
                for (int32_t r = 0; r < run_len; ++r) {
                    const int32_t col = run_start + r, val = V0 - r * u;
                    if (st) {
                        a.fj[er + r] = col;
                        a.fmg[er + r] = pack_mg(val, AE_NEG);
                    } else {
                        a.lj[er + r] = col;
                        a.lM[er + r] = val;
                        a.lGa[er + r] = AE_NEG;
                    }
                    if (st && r < run_hits) {
                        RangeHit rh = {sm.lo[slot], sm.hi[slot], eq, col, val, 0};
                        a.rhits[hr + r] = rh;
                    }
                }
            }
            __syncwarp();
        }
    }
}

template <bool SEQ>
__device__ __forceinline__ void rows_phase(bool write, const DnaRowsArgs &a, WarpSmem &sm, int lane,
                                           unsigned kmask, unsigned smask, uint32_t len, uint64_t noff,
                                           int32_t qm, int32_t qH, int32_t tbase, uint32_t qoff, int32_t qid,
                                           uint32_t woff, uint32_t total) {
    if (SEQ) {
        if (write) rows_seq<true>(a, sm, lane, kmask, smask, len, noff, qm, qH, tbase, qoff, qid);
        else rows_seq<false>(a, sm, lane, kmask, smask, len, noff, qm, qH, tbase, qoff, qid);
    } else {
        if (write) rows_spread<true>(a, sm, lane, kmask, smask, len, noff, qm, qH, tbase, qoff, qid, woff, total);
        else rows_spread<false>(a, sm, lane, kmask, smask, len, noff, qm, qH, tbase, qoff, qid, woff, total);
    }
    __syncwarp();
}

// One launch per level.  Per task: prologue, count phase, reservation of the
// task's output ranges (one atomic per arena on the level's cursors), write
// phase.  A reservation past an arena's capacity leaves the task unwritten and
// raises `retry`; the cursors still advance by every task's totals, so after
// the launch they hold the level's exact sizes either way.
template <bool SEQ>
__global__ void __launch_bounds__(DW * 32, AE_DNA_MINB) k_rows_dna(DnaRowsArgs a) {
    __shared__ WarpSmem smem[DW];
    const int lane = threadIdx.x & 31;
    WarpSmem &sm = smem[threadIdx.x >> 5];
    const int32_t g = a.sc.gmax;
    const int64_t nnodes = a.nnodes;
    const int npt = a.nodes_per_task;
    const uint64_t ntask = (uint64_t)((nnodes + npt - 1) / npt);
    uint64_t trip_mine = 0;   // the (child, parent entry) pairs of this warp's tasks

    for (uint64_t tb = 0;;) {
        if (lane == 0) tb = atomicAdd(&a.ctr->task_c, 4ull);
        tb = __shfl_sync(FULL, tb, 0);
        if (tb >= ntask) break;
    for (uint64_t task = tb; task < tb + 4 && task < ntask; ++task) {
        // ---- prologue: one node per lane
        const int64_t v = (int64_t)task * npt + lane;
        const bool own = lane < npt && v < nnodes;
        Node nd;
        nd.lo = nd.hi = 0;
        nd.item = 0;
        nd.cnt = 0;
        nd.off = 0;
        if (own) nd = a.nodes[v];
        uint32_t clo[4] = {0, 0, 0, 0}, chi[4] = {0, 0, 0, 0};
        unsigned kmask = own ? kids4(a.ix, nd.lo, nd.hi, clo, chi) : 0u;
        const uint32_t len = own ? nd.cnt : 0u;
        if (!len) kmask = 0;
        const int32_t qid = nd.item & 0xFFFFFF;
        const uint32_t pcnt = (uint32_t)nd.item >> 24;   // levels the node has been a single occurrence
        // a child stays in the walk while it has several occurrences, or for the
        // first leaf_delay levels after it became a single occurrence
        unsigned smask = 0;   // children that stay in the trie walk
        if (kmask) {
            const bool young = (int)pcnt + 1 <= a.leaf_delay;
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (((kmask >> c) & 1u) && (young || chi[c] - clo[c] >= 2)) smask |= 1u << c;
        }
        int32_t qm = 1, qH = 1;
        uint32_t qoff = 0;
        if (kmask) {
            qm = a.qv.m[qid];
            qH = a.qv.H[qid];
            qoff = (uint32_t)a.qv.off[qid];
        }
        const int32_t tbase = qH - 1 - (qm - 1) * g;   // thr(j) = max(tbase + j g, 0), Theorem 2
        const uint32_t work = kmask ? len : 0u;
        uint32_t woff = work;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, woff, d);
            if (lane >= d) woff += y;
        }
        const uint32_t total = __shfl_sync(FULL, woff, 31);
        woff -= work;
        if (total == 0) continue;
        trip_mine += reduce_add_u64((uint32_t)__popc(kmask) * len);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            sm.a[lane * 4 + c] = 0;
            sm.h[lane * 4 + c] = 0;
            sm.lo[lane * 4 + c] = clo[c];
            sm.hi[lane * 4 + c] = chi[c];
            sm.sinfo[lane * 4 + c] = 0;
        }
        __syncwarp();

        // ---- count phase: per (node, child) outputs and hits
        rows_phase<SEQ>(false, a, sm, lane, kmask, smask, len, nd.off, qm, qH, tbase, qoff, qid, woff, total);

        // ---- reservation: the task's ranges in the five arenas
        unsigned wmask = kmask;   // the children with any output (the others need no write walk)
        uint32_t cn[4] = {0, 0, 0, 0}, ch[4] = {0, 0, 0, 0};
        uint32_t s_fe = 0, s_le = 0, s_fn = 0, s_ln = 0, s_h = 0;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            if ((kmask >> c) & 1u) {
                cn[c] = sm.a[lane * 4 + c];
                ch[c] = sm.h[lane * 4 + c];
                if (cn[c] == 0 && ch[c] == 0) wmask &= ~(1u << c);
                if ((smask >> c) & 1u) {
                    s_fe += cn[c];
                    s_fn += cn[c] ? 1u : 0u;
                } else {
                    s_le += cn[c];
                    s_ln += cn[c] ? 1u : 0u;
                }
                s_h += ch[c];
            }
            sm.be[lane * 4 + c] = cn[c];
            sm.bh[lane * 4 + c] = ch[c];
        }
        uint64_t tsum[5], base[5];
        uint64_t ex_fe, ex_le, ex_fn, ex_ln, ex_h;
        tsum[0] = reduce_add_u64(s_fe);
        tsum[1] = reduce_add_u64(s_le);
        tsum[4] = reduce_add_u64(s_h);
        {   // node counts: at most 128 a task, both in one scan
            const uint32_t nn = s_fn | (s_ln << 16);
            const uint32_t ex = excl_scan_u32(nn);
            const uint32_t tot = __reduce_add_sync(FULL, nn);
            ex_fn = ex & 0xFFFFu;
            ex_ln = ex >> 16;
            tsum[2] = tot & 0xFFFFu;
            tsum[3] = tot >> 16;
        }
        if (tsum[0] + tsum[1] + tsum[4] <= 0xFFFFFFFFull) {   // the usual case: 32-bit scans
            ex_fe = excl_scan_u32(s_fe);
            ex_le = excl_scan_u32(s_le);
            ex_h = excl_scan_u32(s_h);
        } else {
            ex_fe = excl_scan_u64(s_fe, tsum[0]);
            ex_le = excl_scan_u64(s_le, tsum[1]);
            ex_h = excl_scan_u64(s_h, tsum[4]);
        }
        {
            unsigned long long r[5] = {0, 0, 0, 0, 0};
            if (lane == 0) {
                if (tsum[0]) r[0] = atomicAdd(&a.ctr->fr_ent, (unsigned long long)tsum[0]);
                if (tsum[1]) r[1] = atomicAdd(&a.ctr->lf_ent, (unsigned long long)tsum[1]);
                if (tsum[2]) r[2] = atomicAdd(&a.ctr->fr_node, (unsigned long long)tsum[2]);
                if (tsum[3]) r[3] = atomicAdd(&a.ctr->lf_node, (unsigned long long)tsum[3]);
                if (tsum[4]) r[4] = atomicAdd(&a.ctr->hits, (unsigned long long)tsum[4]);
            }
#pragma unroll
            for (int q = 0; q < 5; ++q) base[q] = __shfl_sync(FULL, r[q], 0);
        }
        if (tsum[0] + tsum[1] + tsum[4] == 0) {   // no child kept anything
            __syncwarp();
            continue;
        }
        // a range past an arena's capacity: the task is not written, the level is
        // run again with arenas of the exact sizes the cursors then hold
        const bool full = base[0] + tsum[0] > a.fr_ent_cap || base[1] + tsum[1] > a.lf_ent_cap ||
                          base[2] + tsum[2] > a.fr_node_cap || base[3] + tsum[3] > a.lf_node_cap ||
                          base[4] + tsum[4] > a.hit_cap;
        if (full) {
            if (lane == 0) atomicExch(&a.ctr->retry, 1ull);
            __syncwarp();
            continue;
        }
        if (lane == 0) {
            sm.base[0] = base[0];
            sm.base[1] = base[1];
            sm.base[2] = base[4];
        }
        uint64_t efr = ex_fe, elf = ex_le, nfr = ex_fn, nlf = ex_ln, hh = ex_h;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            if (!((kmask >> c) & 1u)) continue;
            const bool st = (smask >> c) & 1u;
            const uint64_t e = st ? efr : elf;
            sm.a[lane * 4 + c] = (uint32_t)e;
            sm.h[lane * 4 + c] = (uint32_t)hh;
            if (cn[c]) {
                if (st) {
                    Node cn_;
                    cn_.lo = clo[c];
                    cn_.hi = chi[c];
                    const uint32_t uq = (chi[c] - clo[c] == 1) ? pcnt + 1u : 0u;
                    cn_.item = (int32_t)((uint32_t)qid | (uq << 24));
                    cn_.cnt = cn[c];
                    cn_.off = base[0] + e;
                    a.fnodes[base[2] + nfr] = cn_;
                    ++nfr;
                } else {
                    Inject in;
                    in.qid = qid;
                    in.e = a.ix.tend[clo[c]];
                    in.cnt = cn[c];
                    in.pad = 0;
                    in.off = base[1] + e;
                    a.inj[base[3] + nlf] = in;
                    ++nlf;
                }
            }
            if (st) efr += cn[c];
            else elf += cn[c];
            hh += ch[c];
        }
        __syncwarp();

        // ---- write phase: staged rows are copied to their reserved positions (four
        // slots per lane), the others computed again and written there
        unsigned rmask = wmask;
        if (SEQ && a.stage) {
            const uint2 *wst = a.stage + (int64_t)(blockIdx.x * DW + (threadIdx.x >> 5)) * 32 * a.stage_cap;
#pragma unroll 1
            for (int s0 = 0; s0 < 128; s0 += 32) {
                const int slot = s0 + lane, L = slot >> 2, c = slot & 3;
                const int32_t HL = __shfl_sync(FULL, qH, L), qL = __shfl_sync(FULL, qid, L);
                const unsigned smL = __shfl_sync(FULL, smask, L), wmL = __shfl_sync(FULL, wmask, L);
                const uint32_t info = sm.sinfo[slot];
                if (!((wmL >> c) & 1u) || !(info >> 31)) continue;
                const bool st = (smL >> c) & 1u;
                const uint32_t n = sm.be[slot], nh = sm.bh[slot];
                const uint64_t e = sm.base[st ? 0 : 1] + sm.a[slot];
                const uint64_t h0 = sm.base[2] + sm.h[slot];
                const uint2 *src = wst + (int64_t)((info >> 16) & 31u) * a.stage_cap + (info & 0xFFFFu);
                const uint32_t clo_ = sm.lo[slot], chi_ = sm.hi[slot];
                uint32_t nhit = 0;
                for (uint32_t k = 0; k < n; ++k) {
                    const uint2 x = src[k];
                    const int32_t j = (int32_t)x.x;
                    const int32_t M = mg_lo(x.y);
                    if (st) {
                        a.fj[e + k] = j;
                        a.fmg[e + k] = x.y;
                        if (M >= HL) {   // a kept entry reaching H is a hit (Section 2.2)
                            if (nhit < nh) a.rhits[h0 + nhit] = RangeHit{clo_, chi_, qL, j, M, 0};
                            ++nhit;
                        }
                    } else {
                        a.lj[e + k] = j;
                        a.lM[e + k] = M;
                        a.lGa[e + k] = mg_hi(x.y);
                    }
                }
                if (st && nhit != nh) atomicExch(&a.ctr->overflow, 1ull);   // the phases disagree
            }
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (sm.sinfo[lane * 4 + c] >> 31) rmask &= ~(1u << c);
        }
        if (__any_sync(FULL, rmask != 0))
            rows_phase<SEQ>(true, a, sm, lane, rmask, smask, len, nd.off, qm, qH, tbase, qoff, qid, woff, total);
    }
    }
    if (lane == 0 && trip_mine) atomicAdd(&a.ctr->triples, (unsigned long long)trip_mine);
}


// ---- levels of few nodes with long rows: one block per node
//
// The spread layout gives a node one warp, which carries its row's
// horizontal-gap scan from chunk to chunk; a level of a few hundred nodes with
// rows of thousands of entries then runs on a few hundred warps.  Here a whole
// block takes a node: each chunk of WB_T parent entries is spread one per
// thread, and per child the keys are a block-wide max-scan carried from chunk
// to chunk.  The count phase sums each child's outputs, thread 0 reserves the
// node's ranges (as a task of k_rows_dna does), and the write phase computes
// the chunks again and writes at block-wide exclusive sums of the counts.  The
// values are those of the other layouts.
constexpr int WB_T = 512;
constexpr int WB_W = WB_T / 32;

struct WideNode {
    uint32_t clo[4], chi[4];
    unsigned kmask, smask, wmask;
    int32_t qid, m, H, full;
    uint32_t pcnt, len, qoff;
    uint64_t off;
    uint64_t pos_e[4], pos_h[4];       // write: each child's next entry and hit positions
    unsigned long long cn[4], ch[4];   // count: each child's entries and hits
    int32_t sw[WB_W];                  // block scans: per-warp values
    unsigned long long sw64[WB_W];
};

__device__ __forceinline__ int32_t wb_scan_max(int32_t v, WideNode &w, int32_t &excl, int32_t &total) {
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    int32_t incl = warp_incl_max(v);
    if (lane == 31) w.sw[wi] = incl;
    __syncthreads();
    int32_t pre = AE_KNEG, all = AE_KNEG;
#pragma unroll
    for (int x = 0; x < WB_W; ++x) {
        const int32_t y = w.sw[x];
        if (x < wi) pre = max(pre, y);
        all = max(all, y);
    }
    int32_t ex = __shfl_up_sync(FULL, incl, 1);
    if (lane == 0) ex = AE_KNEG;
    excl = max(pre, ex);
    total = all;
    __syncthreads();
    return max(pre, incl);
}

__device__ __forceinline__ unsigned long long wb_scan_sum(unsigned long long v, WideNode &w, unsigned long long &total) {
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    unsigned long long incl = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned long long y = __shfl_up_sync(FULL, incl, d);
        if (lane >= d) incl += y;
    }
    if (lane == 31) w.sw64[wi] = incl;
    __syncthreads();
    unsigned long long pre = 0, all = 0;
#pragma unroll
    for (int x = 0; x < WB_W; ++x) {
        const unsigned long long y = w.sw64[x];
        if (x < wi) pre += y;
        all += y;
    }
    total = all;
    __syncthreads();
    return pre + incl - v;   // exclusive
}

__global__ void __launch_bounds__(WB_T) k_rows_dna_wide(DnaRowsArgs a) {
    __shared__ WideNode w;
    const ScoreView &sc = a.sc;
    const int32_t u = -sc.ss, oe = sc.sg + sc.ss, g = sc.gmax, sa = sc.sa, sb = sc.sb;
    const int32_t strong = -oe;
    unsigned long long trip_mine = 0;
    for (int64_t v = blockIdx.x; v < a.nnodes; v += gridDim.x) {
        if (threadIdx.x == 0) {
            const Node nd = a.nodes[v];
            uint32_t clo[4] = {0, 0, 0, 0}, chi[4] = {0, 0, 0, 0};
            unsigned kmask = kids4(a.ix, nd.lo, nd.hi, clo, chi);
            if (!nd.cnt) kmask = 0;
            const uint32_t pcnt = (uint32_t)nd.item >> 24;
            unsigned smask = 0;
            if (kmask) {
                const bool young = (int)pcnt + 1 <= a.leaf_delay;
                for (int c = 0; c < 4; ++c)
                    if (((kmask >> c) & 1u) && (young || chi[c] - clo[c] >= 2)) smask |= 1u << c;
            }
            w.qid = nd.item & 0xFFFFFF;
            w.pcnt = pcnt;
            w.len = nd.cnt;
            w.off = nd.off;
            w.kmask = kmask;
            w.smask = smask;
            w.m = kmask ? a.qv.m[w.qid] : 1;
            w.H = kmask ? a.qv.H[w.qid] : 1;
            w.qoff = kmask ? (uint32_t)a.qv.off[w.qid] : 0u;
            w.full = 0;
            for (int c = 0; c < 4; ++c) {
                w.clo[c] = clo[c];
                w.chi[c] = chi[c];
                w.cn[c] = 0;
                w.ch[c] = 0;
            }
        }
        __syncthreads();
        const unsigned kmask = w.kmask, smask = w.smask;
        const uint32_t len = w.len;
        if (!kmask) {
            __syncthreads();
            continue;
        }
        const int32_t m = w.m, H = w.H, qid = w.qid;
        const uint64_t off = w.off;
        const int32_t tb0 = H - 1 - (m - 1) * g;   // thr(j) = max(tb0 + j g, 0), Theorem 2
        const uint8_t *P = a.qv.codes + w.qoff;
        trip_mine += (unsigned long long)__popc(kmask) * len;
        for (int ph = 0; ph < 2; ++ph) {
            const bool write = ph == 1;
            const unsigned pmask = write ? w.wmask : kmask;
            int32_t carry[4] = {AE_KNEG, AE_KNEG, AE_KNEG, AE_KNEG};   // by child index of the phase
            for (uint32_t t0 = 0; t0 < len; t0 += WB_T) {
                const uint32_t t = t0 + threadIdx.x;
                const bool valid = t < len;
                int32_t j = m, jn = m, pjv = -2, pMv = 0;
                uint32_t mg = 0;
                if (valid) {
                    j = a.pj[off + t];
                    mg = a.pmg[off + t];
                    jn = t + 1 < len ? a.pj[off + t + 1] : m;
                    if (t > 0) {
                        pjv = a.pj[off + t - 1];
                        pMv = (int32_t)(int16_t)(a.pmg[off + t - 1] & 0xFFFFu);
                    }
                }
                const bool ok = valid && (uint32_t)j < (uint32_t)m && jn > j && jn <= m;   // a sorted row in [0, m)
                if (valid && !ok) atomicExch(&a.ctr->overflow, 1ull);
                const int32_t M = (int32_t)(int16_t)(mg & 0xFFFFu);
                const bool adjA = ok && pjv + 1 == j && pMv > 0;
                const bool hasB = ok && (j + 1 < m) && (j + 1 != jn);
                const int pA = ok ? (int)P[j] : 255;
                const int pB = hasB ? (int)P[j + 1] : 255;
                const int32_t traw = tb0 + j * g;
                const int32_t tA = max(traw, 0), tB = max(traw + g, 0);
                int32_t Gap = ok ? max((int32_t)(int16_t)(mg >> 16) + sc.ss, M + oe) : AE_NEG;   // dead stays below tA
                Gap = Gap > tA ? Gap : AE_NEG;
                const int32_t ju = j * u;
                unsigned rem = pmask;
#pragma unroll
                for (int i = 0; i < 4; ++i) {   // block-uniform
                    if (!rem) break;
                    const int c = __ffs(rem) - 1;
                    rem &= rem - 1;
                    int32_t MpA = AE_NEG, MpB = AE_NEG;
                    if (ok) {
                        int32_t DA = adjA ? pMv + (c == pA ? sa : sb) : AE_NEG;
                        DA = DA > tA ? DA : AE_NEG;
                        MpA = max(DA, Gap);
                        const int32_t DB = M + (c == pB ? sa : sb);
                        MpB = (hasB && DB > tB) ? DB : AE_NEG;
                    }
                    const int32_t keyA = MpA > strong ? MpA + ju : AE_KNEG;
                    const int32_t keyB = MpB > strong ? MpB + ju + u : AE_KNEG;
                    int32_t excl, tot;
                    int32_t incl = wb_scan_max(max(keyA, keyB), w, excl, tot);
                    excl = max(excl, carry[i]);
                    incl = max(incl, carry[i]);
                    carry[i] = max(carry[i], tot);
                    const int32_t GbA = excl > AE_KNEG / 2 ? sc.sg - ju + excl : AE_NEG;
                    const int32_t MA = max(MpA, GbA);
                    const bool aliveA = ok && MA > tA;
                    int32_t MB = AE_NEG;
                    bool aliveB = false;
                    if (hasB) {
                        const int32_t KB = max(excl, keyA);
                        const int32_t GbB = KB > AE_KNEG / 2 ? sc.sg - ju - u + KB : AE_NEG;
                        MB = max(MpB, GbB);
                        aliveB = MB > tB;
                    }
                    int32_t run_len = 0, run_hits = 0;
                    const int32_t run_start = hasB ? j + 2 : j + 1;
                    const int32_t V0 = sc.sg - run_start * u + incl;
                    if (ok && incl > AE_KNEG / 2 && run_start < jn && V0 > 0) {
                        const int32_t rl = min((int32_t)div_small((uint32_t)(V0 - 1), a.urec) + 1, jn - run_start);
                        if (traw + (run_start + rl - 1) * g <= 0) {
                            run_len = rl;
                            if (V0 >= H) run_hits = min(rl, (int32_t)div_small((uint32_t)(V0 - H), a.urec) + 1);
                        } else {
                            run_of(run_start, jn, incl, sc, m, H, u, run_len, run_hits);
                        }
                    }
                    const bool st = (smask >> c) & 1u;
                    const bool hA = st && aliveA && MA >= H, hB = st && aliveB && MB >= H;
                    const uint32_t cnt = (uint32_t)aliveA + (uint32_t)aliveB + (uint32_t)run_len;
                    const uint32_t hcnt = (uint32_t)hA + (uint32_t)hB + (st ? (uint32_t)run_hits : 0u);
                    if (!write) {
                        // per-warp sums into the child's totals
                        unsigned long long x = ((unsigned long long)cnt << 32) | hcnt;
#pragma unroll
                        for (int d = 16; d > 0; d >>= 1) x += __shfl_down_sync(FULL, x, d);
                        if ((threadIdx.x & 31) == 0 && x) {
                            atomicAdd(&w.cn[c], x >> 32);
                            atomicAdd(&w.ch[c], x & 0xFFFFFFFFull);
                        }
                        continue;
                    }
                    // the child's positions are read before the scan: thread 0 moves them on after it
                    const uint64_t pe = w.pos_e[c], ph = w.pos_h[c];
                    unsigned long long ctot;
                    const unsigned long long ex =
                        wb_scan_sum(((unsigned long long)cnt << 32) | hcnt, w, ctot);
                    uint64_t e0 = pe + (ex >> 32), h0 = ph + (ex & 0xFFFFFFFFull);
                    const uint64_t ecap = st ? a.fr_ent_cap : a.lf_ent_cap;
                    if (cnt && (e0 + cnt > ecap || h0 + hcnt > a.hit_cap)) {   // never past the arenas
                        atomicExch(&a.ctr->overflow, 1ull);
                    } else {
                        const uint32_t clo = w.clo[c], chi = w.chi[c];
                        if (aliveA) {
                            if (st) {
                                a.fj[e0] = j;
                                a.fmg[e0] = pack_mg(MA, Gap);
                            } else {
                                a.lj[e0] = j;
                                a.lM[e0] = MA;
                                a.lGa[e0] = Gap;
                            }
                            ++e0;
                            if (hA) a.rhits[h0++] = RangeHit{clo, chi, qid, j, MA, 0};
                        }
                        if (aliveB) {
                            if (st) {
                                a.fj[e0] = j + 1;
                                a.fmg[e0] = pack_mg(MB, AE_NEG);
                            } else {
                                a.lj[e0] = j + 1;
                                a.lM[e0] = MB;
                                a.lGa[e0] = AE_NEG;
                            }
                            ++e0;
                            if (hB) a.rhits[h0++] = RangeHit{clo, chi, qid, j + 1, MB, 0};
                        }
                        for (int32_t r = 0; r < run_len; ++r) {
                            const int32_t col = run_start + r, val = V0 - r * u;
                            if (st) {
                                a.fj[e0 + r] = col;
                                a.fmg[e0 + r] = pack_mg(val, AE_NEG);
                            } else {
                                a.lj[e0 + r] = col;
                                a.lM[e0 + r] = val;
                                a.lGa[e0 + r] = AE_NEG;
                            }
                            if (st && r < run_hits) a.rhits[h0 + r] = RangeHit{clo, chi, qid, col, val, 0};
                        }
                    }
                    if (threadIdx.x == 0) {
                        w.pos_e[c] += ctot >> 32;
                        w.pos_h[c] += ctot & 0xFFFFFFFFull;
                    }
                    __syncthreads();
                }
            }
            __syncthreads();
            if (!write) {
                // ---- reservation of the node's ranges, as a task of k_rows_dna does
                if (threadIdx.x == 0) {
                    unsigned long long s_fe = 0, s_le = 0, s_fn = 0, s_ln = 0, s_h = 0;
                    unsigned wmask = kmask;
                    for (int c = 0; c < 4; ++c) {
                        if (!((kmask >> c) & 1u)) continue;
                        if (w.cn[c] == 0 && w.ch[c] == 0) wmask &= ~(1u << c);
                        if ((smask >> c) & 1u) {
                            s_fe += w.cn[c];
                            s_fn += w.cn[c] ? 1 : 0;
                        } else {
                            s_le += w.cn[c];
                            s_ln += w.cn[c] ? 1 : 0;
                        }
                        s_h += w.ch[c];
                    }
                    w.wmask = wmask;
                    const unsigned long long b0 = s_fe ? atomicAdd(&a.ctr->fr_ent, s_fe) : 0;
                    const unsigned long long b1 = s_le ? atomicAdd(&a.ctr->lf_ent, s_le) : 0;
                    const unsigned long long b2 = s_fn ? atomicAdd(&a.ctr->fr_node, s_fn) : 0;
                    const unsigned long long b3 = s_ln ? atomicAdd(&a.ctr->lf_node, s_ln) : 0;
                    const unsigned long long b4 = s_h ? atomicAdd(&a.ctr->hits, s_h) : 0;
                    const bool full = (s_fe && b0 + s_fe > a.fr_ent_cap) || (s_le && b1 + s_le > a.lf_ent_cap) ||
                                      (s_fn && b2 + s_fn > a.fr_node_cap) || (s_ln && b3 + s_ln > a.lf_node_cap) ||
                                      (s_h && b4 + s_h > a.hit_cap);
                    w.full = full ? 1 : 0;
                    if (full) {
                        atomicExch(&a.ctr->retry, 1ull);
                    } else {
                        uint64_t efr = b0, elf = b1, nfr = b2, nlf = b3, hh = b4;
                        for (int c = 0; c < 4; ++c) {
                            if (!((kmask >> c) & 1u)) continue;
                            const bool st = (smask >> c) & 1u;
                            w.pos_e[c] = st ? efr : elf;
                            w.pos_h[c] = hh;
                            const uint32_t cn = (uint32_t)w.cn[c];
                            if (cn) {
                                if (st) {
                                    Node cn_;
                                    cn_.lo = w.clo[c];
                                    cn_.hi = w.chi[c];
                                    const uint32_t uq = (w.chi[c] - w.clo[c] == 1) ? w.pcnt + 1u : 0u;
                                    cn_.item = (int32_t)((uint32_t)qid | (uq << 24));
                                    cn_.cnt = cn;
                                    cn_.off = efr;
                                    a.fnodes[nfr++] = cn_;
                                } else {
                                    Inject in;
                                    in.qid = qid;
                                    in.e = a.ix.tend[w.clo[c]];
                                    in.cnt = cn;
                                    in.pad = 0;
                                    in.off = elf;
                                    a.inj[nlf++] = in;
                                }
                            }
                            if (st) efr += cn;
                            else elf += cn;
                            hh += w.ch[c];
                        }
                    }
                }
                __syncthreads();
                if (w.full || !w.wmask) break;   // block-uniform
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && trip_mine) atomicAdd(&a.ctr->triples, trip_mine);
}
}  // namespace

int ae_rows_dna_blocks_per_sm() { return AE_DNA_MINB; }
int ae_rows_dna_warps_per_block() { return DW; }

void ae_rows_dna(const DnaRowsArgs &a, int blocks, cudaStream_t st) {
    if (a.nnodes <= 0) return;
    ++g_launches;
    if (a.sequential == 2) {   // one block per node
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int64_t nb = std::min<int64_t>(a.nnodes, (int64_t)sms * 4);
        k_rows_dna_wide<<<(unsigned)nb, WB_T, 0, st>>>(a);
    } else if (a.sequential)
        k_rows_dna<true><<<blocks, DW * 32, 0, st>>>(a);
    else
        k_rows_dna<false><<<blocks, DW * 32, 0, st>>>(a);
}
