// One level of the breadth-wise suffix-trie walk (Section 5 (3)) with the
// Gotoh rows of Section 2.2, on sm_103a.
//
//   k_children   every (node, letter c) pair: the child's SA range by one
//                backward-search step, lo' = C[c] + Occ(c, lo), hi' = C[c] +
//                Occ(c, hi); a non-empty child inherits its parent's row length
//                as the number of "triples" (child, parent entry) to compute.
//   scan+compact the non-empty children become segments laid end to end, with
//                a table of the first segment of every task window.
//   k_rows       the triples are packed densely into warp lanes (many small
//                rows share one warp); horizontal gaps use segmented max-plus
//                scans.  A count pass counts every task's outputs (and keeps
//                each triple's final slot values); after an exclusive scan of
//                the task totals, a write pass writes the outputs at their
//                offsets.
//
// Children with one occurrence leave the trie: their rows go to the leaf
// arena as injections for the text-position sweep.
#include <cuda_runtime.h>
#include <stdint.h>

#include "ae_device.cuh"
#include "ae_kernels.h"

namespace {
using namespace aedev;

// Child ranges of node nd (Section 5 (3)): one backward-search step per
// letter; a single occurrence has only the child BWT[lo] (one LF step).
// Calls f(letter, lo', hi') for every non-empty child in letter order.
template <int SIGMA, typename F>
__device__ __forceinline__ void for_children(const IndexView &ix, const Node &nd, F f) {
    if (nd.hi - nd.lo == 1) {
        if ((int64_t)nd.lo == ix.dollar_row || sep_row(ix, nd.lo)) return;
        const int b = bwt_letter<SIGMA>(ix, nd.lo);
        const uint32_t lo = ix.C[b] + occ_of<SIGMA>(ix, b, nd.lo);
        f(b, lo, lo + 1);
        return;
    }
    for (int c = 0; c < SIGMA; ++c) {
        const uint32_t lo = ix.C[c] + occ_of<SIGMA>(ix, c, nd.lo);
        const uint32_t hi = ix.C[c] + occ_of<SIGMA>(ix, c, nd.hi);
        if (hi > lo) f(c, lo, hi);
    }
}

__device__ __forceinline__ uint32_t row_len(const ChildrenArgs &a, const Node &nd) {
    if (nd.cnt == AE_ROOT_ROW) {
        const WorkItem it = a.items[nd.item];
        return (uint32_t)(it.c1 - it.c0);
    }
    return nd.cnt;
}

// Per node: how many non-empty children and how many triples (child, parent
// entry) they carry.
template <int SIGMA>
__global__ void k_children(ChildrenArgs a) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < a.nnodes;
         v += (int64_t)gridDim.x * blockDim.x) {
        const Node nd = a.nodes[v];
        const uint32_t len = row_len(a, nd);
        uint32_t nseg = 0;
        for_children<SIGMA>(a.ix, nd, [&](int, uint32_t, uint32_t) { ++nseg; });
        a.nseg[v] = len ? nseg : 0u;
        a.ntrip[v] = len ? nseg * len : 0u;
    }
    if (a.stats && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&a.stats->nodes, (unsigned long long)a.nnodes);
}

// Per node: write its non-empty children as segments at the scanned offsets.
template <int SIGMA>
__global__ void k_compact(ChildrenArgs a, const uint64_t *seg_off, const uint64_t *trip_off, Seg *segs,
                          uint64_t *task_first) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < a.nnodes;
         v += (int64_t)gridDim.x * blockDim.x) {
        const Node nd = a.nodes[v];
        const uint32_t len = row_len(a, nd);
        if (!len) continue;
        const bool root = nd.cnt == AE_ROOT_ROW;
        uint64_t so = seg_off[v], to = trip_off[v];
        // next task window start at or after `to` (one division per node; the
        // segments of a node are consecutive, so later windows follow by adding)
        uint64_t wq = (to + AE_ROW_TASK - 1) / AE_ROW_TASK;
        uint32_t cq_hi;
        uint64_t poff;
        uint32_t len_hi = 0;
        if (root) {
            const WorkItem it = a.items[nd.item];
            cq_hi = ((uint32_t)it.qid << 5) | 0x80000000u;
            poff = (uint64_t)(uint32_t)it.c0 | ((uint64_t)(uint32_t)it.c1 << 32);
        } else {
            // nd.item packs the query id (bits 0-23) and the levels the node has
            // been a single occurrence (bits 24-31)
            cq_hi = ((uint32_t)nd.item & 0xFFFFFFu) << 5;
            len_hi = ((uint32_t)nd.item >> 24) << 28;
            poff = nd.off;
        }
        for_children<SIGMA>(a.ix, nd, [&](int c, uint32_t lo, uint32_t hi) {
            Seg s;
            s.lo = lo;
            s.hi = hi;
            s.len = len | len_hi;
            s.cq = (uint32_t)c | cq_hi;
            s.toff = to;
            s.poff = poff;
            segs[so] = s;
            // task windows that begin inside this segment: the first segment at or
            // after the window start is this one (start on its first triple) or the next
            for (; wq * AE_ROW_TASK < to + len; ++wq) task_first[wq] = wq * AE_ROW_TASK == to ? so : so + 1;
            ++so;
            to += len;
        });
    }
}

// A child stays in the trie walk (instead of going to the text-position
// sweep) while it has several occurrences, or for the first `delay` levels
// after it became a single occurrence: short-lived rows then die here, packed
// many to a warp, and only the long-lived ones reach the sweep, which merges
// rows meeting at one text position.
__device__ __forceinline__ bool seg_stays(const Seg &sg, int delay) {
    if (sg.hi - sg.lo >= 2) return true;
    return (int)(sg.len >> 28) + 1 <= delay;
}

#ifndef AE_RW_WARPS
#define AE_RW_WARPS 8
#endif
constexpr int RW_WARPS = AE_RW_WARPS;
constexpr int RW_TASK = AE_ROW_TASK;   // triples per task window = max segments per task
#ifndef AE_RW_GRAB
#define AE_RW_GRAB 4
#endif
constexpr int RW_GRAB = AE_RW_GRAB;    // tasks per take from the task counter
// Resident blocks per SM the two passes are compiled for (and launched with):
// the kernel is bound by memory latency per triple, so more resident warps
// beat more registers (measured on the 100 Mbp workload: 6 blocks of 8 warps)
#ifndef AE_RW_MINB_COUNT
#define AE_RW_MINB_COUNT 6
#endif
#ifndef AE_RW_MINB_WRITE
#define AE_RW_MINB_WRITE 6
#endif
constexpr int RW_MINB_COUNT = AE_RW_MINB_COUNT, RW_MINB_WRITE = AE_RW_MINB_WRITE;

struct TaskSmem {
    uint32_t cnt[RW_TASK];
    uint32_t hit[RW_TASK];
    uint64_t base[RW_TASK];
    uint64_t hbase[RW_TASK];
};

// Process the triples [t_beg, t_end) of one task, whose segments are
// [s_first, s_last).  Pass 1 (WRITE = false) adds each segment's output and
// hit counts into sm; pass 2 writes entries and hits at sm.base/hbase plus
// the running counts.
//
// With a.res (int16x2 route), the count pass also stores each triple's final
// slot values (M of slot A in the low, of slot B in the high halfword; 0 =
// dead) and its gap-run key, and the write pass is run_task_stored.
template <int SIGMA, bool WRITE, bool I16>
__device__ void run_task(const RowsArgs &a, const int8_t *smat, TaskSmem &sm, uint64_t s_first, uint64_t s_last,
                         uint64_t t_beg, uint64_t t_end, unsigned long long &st0, unsigned long long &st1,
                         unsigned long long &st2, unsigned long long &st_cand, unsigned long long &st_np,
                         unsigned long long &st_nr) {
    const int lane = threadIdx.x & 31;
    const unsigned le = (lane == 31) ? 0xffffffffu : ((1u << (lane + 1)) - 1u);
    const ScoreView &sc = a.sc;
    const int32_t u = -sc.ss, oe = sc.sg + sc.ss, g = sc.gmax;
    // a gap state reached from slot value M' can be live only if M' > |s_g + s_s|
    // (Eq. 3): weaker slots give the G_b scan no key, and a chunk without a key
    // or an incoming carry skips the scan
    const int32_t strong = -oe;
    uint64_t sbase = s_first;
    int32_t carry = AE_KNEG;
    // triple offsets relative to the task (a task spans < 2^32 triples)
    const uint32_t t_len = (uint32_t)(t_end - t_beg);
    for (uint32_t t0 = 0; t0 < t_len; t0 += 32) {
        const uint32_t t = t0 + lane;
        const bool valid = t < t_len;
        const uint32_t woff = (sbase + lane < s_last) ? (uint32_t)(a.segs[sbase + lane].toff - t_beg) : 0xFFFFFFFFu;
        int i = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const uint32_t o = __shfl_sync(FULL, woff, i + step);
            if (o <= t) i += step;
        }
        const uint64_t sid = sbase + i;
        Seg sg;
        sg.len = 0;
        sg.toff = 0;
        sg.poff = 0;
        sg.lo = sg.hi = 0;
        sg.cq = 0;
        if (valid) sg = a.segs[sid];
        const int32_t k = valid ? (int32_t)(t - (uint32_t)(sg.toff - t_beg)) : 0;
        const uint32_t slen = sg.len & 0x0FFFFFFFu;
        const int c = (int)(sg.cq & 31u);
        const int32_t qid = (int32_t)((sg.cq >> 5) & 0xFFFFFFu);
        const bool root = (sg.cq >> 31) != 0;
        int32_t m = 1, H = 1;
        const uint8_t *P = a.qv.codes;
        if (valid) {
            m = a.qv.m[qid];
            H = a.qv.H[qid];
            P += a.qv.off[qid];
        }
        // ---- slots of this lane (see slot_finish)
        int32_t colA = m, MpA = AE_NEG, GaA = AE_NEG, MpB = AE_NEG, next_col = m;
        int32_t Dprev = AE_NEG, Gap = AE_NEG, Dk = AE_NEG, Gap_raw = AE_NEG;
        bool hasB = false;
        const unsigned heads = __ballot_sync(FULL, !valid || k == 0 || lane == 0);
        const int first_lane = 31 - __clz(heads & le);
        // neighbours inside the segment
        int32_t j = m, M = AE_NEG, Ga = AE_NEG;
        uint32_t mg = 0;
        if (valid && !root) {
            j = a.pj[sg.poff + k];
            if (I16) {
                mg = reinterpret_cast<const uint32_t *>(a.pM)[sg.poff + k];
                M = mg_lo(mg);
            } else {
                M = a.pM[sg.poff + k];
                Ga = a.pGa[sg.poff + k];
            }
        }
        int32_t jn = __shfl_down_sync(FULL, j, 1);
        int32_t pjv = __shfl_up_sync(FULL, j, 1), pMv = __shfl_up_sync(FULL, M, 1);
        if (valid && !root) {
            const bool next_in = (lane < 31) && (((heads >> (lane + 1)) & 1u) == 0);
            if (!next_in) jn = ((uint32_t)k + 1 < slen) ? a.pj[sg.poff + k + 1] : m;
            if (lane == first_lane) {   // first lane of its segment in this chunk
                if (k > 0) {
                    pjv = a.pj[sg.poff + k - 1];
                    pMv = I16 ? mg_lo(reinterpret_cast<const uint32_t *>(a.pM)[sg.poff + k - 1])
                              : a.pM[sg.poff + k - 1];
                } else {
                    pjv = -2;
                    pMv = AE_NEG;
                }
            }
        }
        if (valid) {
            if (root) {
                const int32_t c0 = (int32_t)(uint32_t)sg.poff, c1 = (int32_t)(uint32_t)(sg.poff >> 32);
                colA = c0 + (int32_t)k;
                const int32_t D = delta_of(sc, smat, c, P[colA]);
                // a search split over ranks opens forks only at its own start columns
                const bool mine = a.parts <= 1 || colA % a.parts == a.part;
                Dprev = (mine && D > thr_of(colA, m, H, g)) ? D : AE_NEG;
                MpA = Dprev;
                next_col = (colA + 1 < c1) ? colA + 1 : m;
            } else {
                colA = j;
                const int32_t tA = thr_of(j, m, H, g);
                if (pjv + 1 == j && pMv > AE_NEG) {
                    const int32_t D = pMv + delta_of(sc, smat, c, P[j]);
                    Dprev = D > tA ? D : AE_NEG;
                }
                const int32_t gap = I16 ? gap_from_mg(mg, sc.ss, oe) : gap_from_i32(M, Ga, sc.ss, oe);
                Gap_raw = gap;
                Gap = gap > tA ? gap : AE_NEG;
                MpA = max(Dprev, Gap);
                GaA = Gap;
                hasB = (j + 1 < m) && (j + 1 != jn);
                if (hasB) {
                    const int32_t D = M + delta_of(sc, smat, c, P[j + 1]);
                    Dk = D > thr_of(j + 1, m, H, g) ? D : AE_NEG;
                    MpB = Dk;
                }
                next_col = jn;
            }
        }
        // ---- segmented max-plus scan of the keys M'(k) + k*u of strong slots
        const int32_t keyA = MpA > strong ? MpA + colA * u : AE_KNEG;
        const int32_t keyB = MpB > strong ? MpB + (colA + 1) * u : AE_KNEG;
        int32_t incl = max(keyA, keyB);
        const int32_t k0 = __shfl_sync(FULL, k, 0);
        const bool cont = (first_lane == 0) && valid && k0 > 0;   // segment continues from the last chunk
        int32_t excl = AE_KNEG;
        if (__any_sync(FULL, incl > AE_KNEG || (cont && carry > AE_KNEG))) {
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int32_t o = __shfl_up_sync(FULL, incl, d);
                if (lane - d >= first_lane) incl = max(incl, o);
            }
            if (cont) incl = max(incl, carry);
            excl = __shfl_up_sync(FULL, incl, 1);
            if (lane - 1 < first_lane) excl = cont ? carry : AE_KNEG;
        }
        SlotOut o;
        slot_finish(colA, MpA, hasB, MpB, next_col, excl, incl, sc, m, H, u, valid, o);
        {
            const uint32_t k31 = (uint32_t)__shfl_sync(FULL, k, 31);
            const bool v31 = __shfl_sync(FULL, valid, 31);
            const uint32_t len31 = __shfl_sync(FULL, slen, 31);
            const int32_t inc31 = __shfl_sync(FULL, incl, 31);
            const bool goes_on = v31 && (k31 + 1 < len31);
            carry = goes_on ? inc31 : AE_KNEG;
            const uint64_t sid31 = __shfl_sync(FULL, sid, 31);
            sbase = goes_on ? sid31 : sid31 + 1;
        }

        // ---- counts, segmented sums
        const bool kind1 = valid && seg_stays(sg, a.leaf_delay);
        const uint32_t nA = o.aliveA, nB = o.aliveB, nR = (uint32_t)o.run_len;
        const uint32_t cnt = nA + nB + nR;
        const uint32_t hA = o.aliveA && o.MA >= H, hB = o.aliveB && o.MB >= H;
        const uint32_t hcnt = kind1 ? (hA + hB + (uint32_t)o.run_hits) : 0u;
        // segmented inclusive sums of cnt and hcnt: without a run in the chunk every
        // term is a 0/1 flag and the sums are population counts of ballots
        uint32_t ci = cnt, hi = hcnt;
        if (__any_sync(FULL, nR > 0)) {
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t oc = __shfl_up_sync(FULL, ci, d), oh = __shfl_up_sync(FULL, hi, d);
                if (lane - d >= first_lane) {
                    ci += oc;
                    hi += oh;
                }
            }
        } else {
            const unsigned in_seg = le & ~((1u << first_lane) - 1u);     // lanes first_lane..lane
            const unsigned bA = __ballot_sync(FULL, o.aliveA), bB = __ballot_sync(FULL, o.aliveB);
            const unsigned bhA = __ballot_sync(FULL, kind1 && hA), bhB = __ballot_sync(FULL, kind1 && hB);
            ci = __popc(bA & in_seg) + __popc(bB & in_seg);
            hi = __popc(bhA & in_seg) + __popc(bhB & in_seg);
        }
        const bool is_last = valid && (lane == 31 || ((heads >> (lane + 1)) & 1u));
        const uint64_t rel = sid - s_first;
        if (!WRITE) {
            if (is_last) {
                sm.cnt[rel] += ci;
                sm.hit[rel] += hi;
            }
            if (I16 && a.res && valid) {
                a.res[t_beg + t] = (o.aliveA ? (uint32_t)o.MA : 0u) | ((o.aliveB ? (uint32_t)o.MB : 0u) << 16);
                a.res_key[t_beg + t] = o.run_len > 0 ? incl : AE_KNEG;
            }
            __syncwarp();
            continue;
        }
        // ---- write entries (and hits of multi-occurrence children)
        const bool overflow_task = false;
        (void)overflow_task;
        uint64_t e0 = 0, h0 = 0;
        int32_t *oj = nullptr, *oM = nullptr, *oGa = nullptr;
        // frontier rows of the int16 route are packed pairs (oGa = null)
        const bool packed = I16 && kind1;
        if (valid) {
            e0 = sm.base[rel] + sm.cnt[rel] + (ci - cnt);
            h0 = sm.hbase[rel] + sm.hit[rel] + (hi - hcnt);
            if (kind1) {
                oj = a.fj;
                oM = a.fM;
                oGa = I16 ? nullptr : a.fGa;
            } else {
                oj = a.lj;
                oM = a.lM;
                oGa = a.lGa;
            }
        }
        __syncwarp();
        if (is_last) {
            sm.cnt[rel] += ci;
            sm.hit[rel] += hi;
        }
        if (o.aliveA) {
            oj[e0] = colA;
            if (packed) {
                reinterpret_cast<uint32_t *>(oM)[e0] = pack_mg(o.MA, GaA);
            } else {
                oM[e0] = o.MA;
                oGa[e0] = GaA;
            }
            if (a.tiers) {
                const int tier = (Dprev > AE_NEG) + (Gap > AE_NEG) + (o.GbA > thr_of(colA, m, H, g));
                st0 += tier <= 1;
                st1 += tier == 2;
                st2 += tier == 3;
            }
        }
        if (o.aliveB) {
            oj[e0 + nA] = colA + 1;
            if (packed) {
                reinterpret_cast<uint32_t *>(oM)[e0 + nA] = pack_mg(o.MB, AE_NEG);
            } else {
                oM[e0 + nA] = o.MB;
                oGa[e0 + nA] = AE_NEG;
            }
            if (a.tiers) {
                const int tier = (Dk > AE_NEG) + (o.GbB > thr_of(colA + 1, m, H, g));
                st0 += tier <= 1;
                st1 += tier == 2;
            }
        }
        if (a.tiers) {
            st0 += nR;
            // filter statistics (Theorem 2): the slot candidates of this triple and
            // those dropped as non-positive or as unable to reach H
            if (valid) {
                const int32_t tA = thr_of(colA, m, H, g);
                int32_t vA = max(Gap_raw, o.GbA);
                if (!root && pjv + 1 == j && pMv > AE_NEG) vA = max(vA, pMv + delta_of(sc, smat, c, P[j]));
                if (root) vA = max(vA, delta_of(sc, smat, c, P[colA]));
                unsigned long long cand = 1, np = vA <= 0, nr = vA > 0 && vA <= tA;
                if (hasB) {
                    const int32_t vB = max(M + delta_of(sc, smat, c, P[j + 1]), o.GbB);
                    cand += 1;
                    np += vB <= 0;
                    nr += vB > 0 && vB <= thr_of(colA + 1, m, H, g);
                }
                st_cand += cand;
                st_np += np;
                st_nr += nr;
            }
        }
        if (kind1) {
            uint64_t hp = h0;
            if (hA) {
                RangeHit r = {sg.lo, sg.hi, qid, colA, o.MA, 0};
                a.rhits[hp++] = r;
            }
            if (hB) {
                RangeHit r = {sg.lo, sg.hi, qid, colA + 1, o.MB, 0};
                a.rhits[hp++] = r;
            }
        }
        unsigned rmask = __ballot_sync(FULL, nR > 0);
        while (rmask) {
            const int L = __ffs(rmask) - 1;
            rmask &= rmask - 1;
            const int32_t s0 = __shfl_sync(FULL, o.run_start, L);
            const int32_t rl = __shfl_sync(FULL, o.run_len, L);
            const int32_t rh = __shfl_sync(FULL, o.run_hits, L);
            const int32_t K = __shfl_sync(FULL, incl, L);
            const uint64_t d0 = __shfl_sync(FULL, e0 + nA + nB, L);
            const uint64_t hd = __shfl_sync(FULL, h0 + hA + hB, L);
            const bool k1 = __shfl_sync(FULL, kind1, L);
            int32_t *rj = (int32_t *)__shfl_sync(FULL, (unsigned long long)oj, L);
            int32_t *rM = (int32_t *)__shfl_sync(FULL, (unsigned long long)oM, L);
            int32_t *rG = (int32_t *)__shfl_sync(FULL, (unsigned long long)oGa, L);
            const uint32_t rlo = __shfl_sync(FULL, sg.lo, L), rhi = __shfl_sync(FULL, sg.hi, L);
            const int32_t rq = __shfl_sync(FULL, qid, L);
            for (int32_t tt = lane; tt < rl; tt += 32) {
                const int32_t col = s0 + tt;
                const int32_t v = sc.sg - col * u + K;
                rj[d0 + tt] = col;
                if (rG) {
                    rM[d0 + tt] = v;
                    rG[d0 + tt] = AE_NEG;
                } else {
                    reinterpret_cast<uint32_t *>(rM)[d0 + tt] = pack_mg(v, AE_NEG);
                }
                if (k1 && tt < rh) {
                    RangeHit r = {rlo, rhi, rq, col, v, 0};
                    a.rhits[hd + tt] = r;
                }
            }
        }
        __syncwarp();
    }
}

// Write pass from the slot values the count pass stored (int16x2 route): the
// same outputs at the same places as run_task with WRITE, without recomputing
// the recurrence.  G_a of slot A is the vertical gap of the parent entry
// (Section 2.2), recomputed from the parent; a gap run is rebuilt in closed
// form from its stored key K (run_of).
template <int SIGMA>
__device__ void run_task_stored(const RowsArgs &a, TaskSmem &sm, uint64_t s_first, uint64_t s_last,
                                uint64_t t_beg, uint64_t t_end) {
    const int lane = threadIdx.x & 31;
    const unsigned le = (lane == 31) ? 0xffffffffu : ((1u << (lane + 1)) - 1u);
    const ScoreView &sc = a.sc;
    const int32_t oe = sc.sg + sc.ss, g = sc.gmax;
    uint64_t sbase = s_first;
    const uint32_t t_len = (uint32_t)(t_end - t_beg);
    for (uint32_t t0 = 0; t0 < t_len; t0 += 32) {
        const uint32_t t = t0 + lane;
        const bool valid = t < t_len;
        const uint32_t woff = (sbase + lane < s_last) ? (uint32_t)(a.segs[sbase + lane].toff - t_beg) : 0xFFFFFFFFu;
        int i = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const uint32_t o = __shfl_sync(FULL, woff, i + step);
            if (o <= t) i += step;
        }
        const uint64_t sid = sbase + i;
        Seg sg;
        sg.len = 0;
        sg.toff = 0;
        sg.poff = 0;
        sg.lo = sg.hi = 0;
        sg.cq = 0;
        if (valid) sg = a.segs[sid];
        const int32_t k = valid ? (int32_t)(t - (uint32_t)(sg.toff - t_beg)) : 0;
        const uint32_t slen = sg.len & 0x0FFFFFFFu;
        const int32_t qid = (int32_t)((sg.cq >> 5) & 0xFFFFFFu);
        const bool root = (sg.cq >> 31) != 0;
        const unsigned heads = __ballot_sync(FULL, !valid || k == 0 || lane == 0);
        const int first_lane = 31 - __clz(heads & le);
        const uint32_t w = valid ? a.res[t_beg + t] : 0u;
        const int32_t K = valid ? a.res_key[t_beg + t] : AE_KNEG;
        const int32_t MA = (int32_t)(w & 0xFFFFu), MB = (int32_t)(w >> 16);
        const bool aliveA = MA > 0, aliveB = MB > 0;
        int32_t colA = 0, GaA = AE_NEG, H = 1, m = 1;
        if (valid) {
            H = a.qv.H[qid];
            m = a.qv.m[qid];
            if (root) {
                colA = (int32_t)(uint32_t)sg.poff + k;
            } else {
                colA = a.pj[sg.poff + k];
                if (aliveA) {
                    const uint32_t mg = reinterpret_cast<const uint32_t *>(a.pM)[sg.poff + k];
                    const int32_t gap = gap_from_mg(mg, sc.ss, oe);
                    GaA = gap > thr_of(colA, m, H, g) ? gap : AE_NEG;
                }
            }
        }
        // gap run after the lane's slots (rare): rebuild its extent from K
        int32_t run_start = 0, run_len = 0, run_hits = 0;
        const bool chunk_runs = __any_sync(FULL, K > AE_KNEG / 2);
        if (chunk_runs) {
            // next parent column, as run_task derives it
            int32_t jn = __shfl_down_sync(FULL, colA, 1);
            const bool next_in = (lane < 31) && (((heads >> (lane + 1)) & 1u) == 0);
            if (valid && !next_in) {
                if (root) jn = m;
                else jn = ((uint32_t)k + 1 < slen) ? a.pj[sg.poff + k + 1] : m;
            }
            int32_t next_col = m;
            bool hasB = false;
            if (valid) {
                if (root) {
                    const int32_t c1 = (int32_t)(uint32_t)(sg.poff >> 32);
                    next_col = (colA + 1 < c1) ? colA + 1 : m;
                } else {
                    hasB = (colA + 1 < m) && (colA + 1 != jn);
                    next_col = jn;
                }
            }
            run_start = hasB ? colA + 2 : colA + 1;
            run_of(run_start, next_col, K, sc, m, H, -sc.ss, run_len, run_hits);
        }
        {
            const uint32_t k31 = (uint32_t)__shfl_sync(FULL, k, 31);
            const bool v31 = __shfl_sync(FULL, valid, 31);
            const uint32_t len31 = __shfl_sync(FULL, slen, 31);
            const uint64_t sid31 = __shfl_sync(FULL, sid, 31);
            sbase = (v31 && k31 + 1 < len31) ? sid31 : sid31 + 1;
        }
        const bool kind1 = valid && seg_stays(sg, a.leaf_delay);
        const uint32_t nA = aliveA, nB = aliveB, nR = (uint32_t)run_len;
        const uint32_t cnt = nA + nB + nR;
        const uint32_t hA = aliveA && MA >= H, hB = aliveB && MB >= H;
        const uint32_t hcnt = kind1 ? (hA + hB + (uint32_t)run_hits) : 0u;
        uint32_t ci = cnt, hi = hcnt;
        if (chunk_runs) {
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t oc = __shfl_up_sync(FULL, ci, d), oh = __shfl_up_sync(FULL, hi, d);
                if (lane - d >= first_lane) {
                    ci += oc;
                    hi += oh;
                }
            }
        } else {
            const unsigned in_seg = le & ~((1u << first_lane) - 1u);
            const unsigned bA = __ballot_sync(FULL, aliveA), bB = __ballot_sync(FULL, aliveB);
            const unsigned bhA = __ballot_sync(FULL, kind1 && hA), bhB = __ballot_sync(FULL, kind1 && hB);
            ci = __popc(bA & in_seg) + __popc(bB & in_seg);
            hi = __popc(bhA & in_seg) + __popc(bhB & in_seg);
        }
        const bool is_last = valid && (lane == 31 || ((heads >> (lane + 1)) & 1u));
        const uint64_t rel = sid - s_first;
        uint64_t e0 = 0, h0 = 0;
        int32_t *oj = nullptr, *oM = nullptr, *oGa = nullptr;
        if (valid) {
            e0 = sm.base[rel] + sm.cnt[rel] + (ci - cnt);
            h0 = sm.hbase[rel] + sm.hit[rel] + (hi - hcnt);
            if (kind1) {
                oj = a.fj;
                oM = a.fM;
            } else {
                oj = a.lj;
                oM = a.lM;
                oGa = a.lGa;
            }
        }
        __syncwarp();
        if (is_last) {
            sm.cnt[rel] += ci;
            sm.hit[rel] += hi;
        }
        if (aliveA) {
            oj[e0] = colA;
            if (kind1) {
                reinterpret_cast<uint32_t *>(oM)[e0] = pack_mg(MA, GaA);
            } else {
                oM[e0] = MA;
                oGa[e0] = GaA;
            }
        }
        if (aliveB) {
            oj[e0 + nA] = colA + 1;
            if (kind1) {
                reinterpret_cast<uint32_t *>(oM)[e0 + nA] = pack_mg(MB, AE_NEG);
            } else {
                oM[e0 + nA] = MB;
                oGa[e0 + nA] = AE_NEG;
            }
        }
        if (kind1) {
            uint64_t hp = h0;
            if (hA) {
                RangeHit r = {sg.lo, sg.hi, qid, colA, MA, 0};
                a.rhits[hp++] = r;
            }
            if (hB) {
                RangeHit r = {sg.lo, sg.hi, qid, colA + 1, MB, 0};
                a.rhits[hp++] = r;
            }
        }
        if (chunk_runs) {
            unsigned rmask = __ballot_sync(FULL, nR > 0);
            while (rmask) {
                const int L = __ffs(rmask) - 1;
                rmask &= rmask - 1;
                const int32_t s0 = __shfl_sync(FULL, run_start, L);
                const int32_t rl = __shfl_sync(FULL, run_len, L);
                const int32_t rh = __shfl_sync(FULL, run_hits, L);
                const int32_t KL = __shfl_sync(FULL, K, L);
                const uint64_t d0 = __shfl_sync(FULL, e0 + nA + nB, L);
                const uint64_t hd = __shfl_sync(FULL, h0 + hA + hB, L);
                const bool k1 = __shfl_sync(FULL, kind1, L);
                int32_t *rj = (int32_t *)__shfl_sync(FULL, (unsigned long long)oj, L);
                int32_t *rM = (int32_t *)__shfl_sync(FULL, (unsigned long long)oM, L);
                int32_t *rG = (int32_t *)__shfl_sync(FULL, (unsigned long long)oGa, L);
                const uint32_t rlo = __shfl_sync(FULL, sg.lo, L), rhi = __shfl_sync(FULL, sg.hi, L);
                const int32_t rq = __shfl_sync(FULL, qid, L);
                for (int32_t tt = lane; tt < rl; tt += 32) {
                    const int32_t col = s0 + tt;
                    const int32_t v = sc.sg + sc.ss * col + KL;   // s_g - col*u + K
                    rj[d0 + tt] = col;
                    if (k1) {
                        reinterpret_cast<uint32_t *>(rM)[d0 + tt] = pack_mg(v, AE_NEG);
                    } else {
                        rM[d0 + tt] = v;
                        rG[d0 + tt] = AE_NEG;
                    }
                    if (k1 && tt < rh) {
                        RangeHit r = {rlo, rhi, rq, col, v, 0};
                        a.rhits[hd + tt] = r;
                    }
                }
            }
        }
        __syncwarp();
    }
}

// One row pass over all triples.  WRITE = false: every task counts its
// segments' outputs into seg_cnt/seg_hit, its totals per arena into task_tot,
// and the level totals (so the host can size the next arenas exactly); on the
// int16x2 route it also stores each triple's slot values and run key.
// WRITE = true: every task takes its output ranges from the scanned task
// totals (or, after a task total too wide for the scan, from one atomic per
// arena), writes the child node / injection records, and writes the rows and
// the hits of multi-occurrence children, from the stored values or by
// recomputing them.
template <int SIGMA, bool WRITE, bool I16>
__global__ void __launch_bounds__(RW_WARPS * 32, WRITE ? RW_MINB_WRITE : RW_MINB_COUNT) k_rows(RowsArgs a) {
    __shared__ int8_t smat[AE_MAX_SIGMA * AE_MAX_SIGMA];
    __shared__ TaskSmem smem[RW_WARPS];
    load_matrix(a.sc, smat);
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    TaskSmem &sm = smem[wib];
    const uint64_t S = *a.nseg_dev, T = *a.ntrip_dev;
    const uint64_t W = RW_TASK;
    const uint64_t ntask = (T + W - 1) / W;
    unsigned long long st0 = 0, st1 = 0, st2 = 0;
    unsigned long long st_cand = 0, st_np = 0, st_nr = 0;
    unsigned long long st_ent = 0;
    unsigned long long *task_ctr = WRITE ? &a.ctr->task_w : &a.ctr->task_c;
    uint64_t tot_c[5] = {0, 0, 0, 0, 0};    // count pass: this warp's level totals
    // tasks are taken RW_GRAB at a time: one atomic on the shared counter per grab
    for (uint64_t tb = 0;;) {
        if (lane == 0) tb = atomicAdd(task_ctr, (unsigned long long)RW_GRAB);
        tb = __shfl_sync(FULL, tb, 0);
        if (tb >= ntask) break;
    for (uint64_t task = tb; task < tb + RW_GRAB && task < ntask; ++task) {
        const uint64_t s_first = a.task_first[task];
        const uint64_t s_last = task + 1 < ntask ? a.task_first[task + 1] : S;
        if (s_first >= s_last) {
            if (!WRITE && lane < 5) a.task_tot[lane * a.task_stride + task] = 0u;
            continue;
        }
        const uint64_t nsg = s_last - s_first;
        const Seg lastseg = a.segs[s_last - 1];
        const uint64_t t_beg = a.segs[s_first].toff, t_end = lastseg.toff + (lastseg.len & 0x0FFFFFFFu);
        if (!WRITE) {
            for (uint64_t r = lane; r < nsg; r += 32) {
                sm.cnt[r] = 0;
                sm.hit[r] = 0;
            }
            __syncwarp();
            run_task<SIGMA, false, I16>(a, smat, sm, s_first, s_last, t_beg, t_end, st0, st1, st2, st_cand, st_np,
                                        st_nr);
            __syncwarp();
        } else {
            for (uint64_t r = lane; r < nsg; r += 32) {
                sm.cnt[r] = a.seg_cnt[s_first + r];
                sm.hit[r] = a.seg_hit[s_first + r];
            }
            __syncwarp();
        }
        // ---- per-kind totals and exclusive prefixes in segment order.  Per-segment
        // counts of one group of 32 fit 32-bit sums unless a segment holds more than
        // 2^24 outputs (a long gap run); such groups take 64-bit shuffles.
        uint64_t acc[5] = {0, 0, 0, 0, 0};   // fr_ent, lf_ent, fr_node, lf_node, hits
        for (uint64_t r0 = 0; r0 < nsg; r0 += 32) {
            const uint64_t r = r0 + lane;
            uint32_t v[5] = {0, 0, 0, 0, 0};
            bool k1 = false;
            if (r < nsg) {
                const Seg sg = a.segs[s_first + r];
                k1 = seg_stays(sg, a.leaf_delay);
                const uint32_t cn = sm.cnt[r];
                v[0] = k1 ? cn : 0u;
                v[1] = k1 ? 0u : cn;
                v[2] = (k1 && cn) ? 1u : 0u;
                v[3] = (!k1 && cn) ? 1u : 0u;
                v[4] = sm.hit[r];
                if (!WRITE) {
                    a.seg_cnt[s_first + r] = cn;
                    a.seg_hit[s_first + r] = sm.hit[r];
                }
            }
            const bool big = __any_sync(FULL, v[0] > (1u << 24) || v[1] > (1u << 24) || v[4] > (1u << 24));
            if (!WRITE && !big) {
#pragma unroll
                for (int q = 0; q < 5; ++q) acc[q] += __reduce_add_sync(FULL, v[q]);
                continue;
            }
            uint64_t ex[5];
            if (!big) {
                const unsigned before = (1u << lane) - 1u;
                const unsigned b2 = __ballot_sync(FULL, v[2]), b3 = __ballot_sync(FULL, v[3]);
                ex[2] = acc[2] + __popc(b2 & before);
                ex[3] = acc[3] + __popc(b3 & before);
                acc[2] += __popc(b2);
                acc[3] += __popc(b3);
#pragma unroll
                for (int q = 0; q < 5; q += (q == 1 ? 3 : 1)) {   // q = 0, 1, 4
                    uint32_t x = v[q];
#pragma unroll
                    for (int d = 1; d < 32; d <<= 1) {
                        const uint32_t y = __shfl_up_sync(FULL, x, d);
                        if (lane >= d) x += y;
                    }
                    ex[q] = acc[q] + (x - v[q]);
                    acc[q] += __shfl_sync(FULL, x, 31);
                }
            } else {
#pragma unroll
                for (int q = 0; q < 5; ++q) {
                    uint64_t x = v[q];
#pragma unroll
                    for (int d = 1; d < 32; d <<= 1) {
                        const uint64_t y = __shfl_up_sync(FULL, x, d);
                        if (lane >= d) x += y;
                    }
                    ex[q] = acc[q] + x - v[q];
                    acc[q] += __shfl_sync(FULL, x, 31);
                }
            }
            if (WRITE && r < nsg) {
                sm.base[r] = k1 ? ex[0] : ex[1];
                sm.hbase[r] = ex[4] | ((uint64_t)(k1 ? ex[2] : ex[3]) << 40);
            }
        }
        if (!WRITE) {
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                tot_c[q] += acc[q];
                if (lane == q) {
                    a.task_tot[q * a.task_stride + task] = (uint32_t)acc[q];
                    if (acc[q] > 0xFFFFFFFFull) atomicExch(&a.ctr->wide, 1ull);
                }
            }
            st_ent += acc[0] + acc[1];
            continue;
        }
        // output ranges of this task: the scanned count-pass totals, or (after a
        // task total too wide for the scan) one atomic reservation per arena
        unsigned long long b[5] = {0, 0, 0, 0, 0};
        if (a.task_off) {
#pragma unroll
            for (int q = 0; q < 5; ++q) b[q] = a.base_off[q] + a.task_off[q * a.task_stride + task];
        } else {
            if (lane == 0) {
                b[0] = atomicAdd(&a.ctr->fr_ent, (unsigned long long)acc[0]);
                b[1] = atomicAdd(&a.ctr->lf_ent, (unsigned long long)acc[1]);
                b[2] = atomicAdd(&a.ctr->fr_node, (unsigned long long)acc[2]);
                b[3] = atomicAdd(&a.ctr->lf_node, (unsigned long long)acc[3]);
                b[4] = atomicAdd(&a.ctr->hits, (unsigned long long)acc[4]);
            }
#pragma unroll
            for (int q = 0; q < 5; ++q) b[q] = __shfl_sync(FULL, b[q], 0);
        }
        // the count pass sized every arena exactly; a reservation past the end
        // means the two passes disagreed, which is reported, never written
        const bool ovf = b[0] + acc[0] > a.fr_ent_cap || b[1] + acc[1] > a.lf_ent_cap ||
                         b[2] + acc[2] > a.fr_node_cap || b[3] + acc[3] > a.lf_node_cap || b[4] + acc[4] > a.hit_cap;
        if (ovf) {
            if (lane == 0) atomicExch(&a.ctr->overflow, 1ull);
            continue;
        }
        __syncwarp();
        for (uint64_t r = lane; r < nsg; r += 32) {
            const Seg sg = a.segs[s_first + r];
            const bool k1 = seg_stays(sg, a.leaf_delay);
            const uint32_t cn = sm.cnt[r];
            const uint64_t nodeix = sm.hbase[r] >> 40;
            const uint64_t hx = sm.hbase[r] & ((1ull << 40) - 1);
            const uint64_t base = (k1 ? b[0] : b[1]) + sm.base[r];
            sm.base[r] = base;
            sm.hbase[r] = b[4] + hx;
            if (cn) {
                if (k1) {
                    Node cn_;
                    cn_.lo = sg.lo;
                    cn_.hi = sg.hi;
                    // query id, and how many levels the child has been a single occurrence
                    const uint32_t uq = (sg.hi - sg.lo == 1) ? (sg.len >> 28) + 1u : 0u;
                    cn_.item = (int32_t)(((sg.cq >> 5) & 0xFFFFFFu) | (uq << 24));
                    cn_.cnt = cn;
                    cn_.off = base;
                    a.fnodes[b[2] + nodeix] = cn_;
                } else {
                    Inject in;
                    in.qid = (int32_t)((sg.cq >> 5) & 0xFFFFFFu);
                    in.e = a.ix.tend[sg.lo];
                    in.cnt = cn;
                    in.pad = 0;
                    in.off = base;
                    a.inj[b[3] + nodeix] = in;
                }
            }
            sm.cnt[r] = 0;
            sm.hit[r] = 0;
        }
        __syncwarp();
        if (I16 && a.res)
            run_task_stored<SIGMA>(a, sm, s_first, s_last, t_beg, t_end);
        else
            run_task<SIGMA, true, I16>(a, smat, sm, s_first, s_last, t_beg, t_end, st0, st1, st2, st_cand, st_np,
                                       st_nr);
        __syncwarp();
    }
    }
    if (!WRITE && lane == 0) {
        if (tot_c[0]) atomicAdd(&a.ctr->c_fr_ent, (unsigned long long)tot_c[0]);
        if (tot_c[1]) atomicAdd(&a.ctr->c_lf_ent, (unsigned long long)tot_c[1]);
        if (tot_c[2]) atomicAdd(&a.ctr->c_fr_node, (unsigned long long)tot_c[2]);
        if (tot_c[3]) atomicAdd(&a.ctr->c_lf_node, (unsigned long long)tot_c[3]);
        if (tot_c[4]) atomicAdd(&a.ctr->c_hits, (unsigned long long)tot_c[4]);
    }
    if (a.stats) {
        unsigned long long t0 = st0, t1 = st1, t2 = st2, tc = st_cand, tn = st_np, tr = st_nr;
        for (int d = 16; d > 0; d >>= 1) {
            t0 += __shfl_down_sync(FULL, t0, d);
            t1 += __shfl_down_sync(FULL, t1, d);
            t2 += __shfl_down_sync(FULL, t2, d);
            tc += __shfl_down_sync(FULL, tc, d);
            tn += __shfl_down_sync(FULL, tn, d);
            tr += __shfl_down_sync(FULL, tr, d);
        }
        if (lane == 0) {
            if (st_ent) atomicAdd(&a.stats->entries, st_ent);
            if (t0) atomicAdd(&a.stats->tier[0], t0);
            if (t1) atomicAdd(&a.stats->tier[1], t1);
            if (t2) atomicAdd(&a.stats->tier[2], t2);
            if (tc) atomicAdd(&a.stats->cand, tc);
            if (tn) atomicAdd(&a.stats->pruned_nonpos, tn);
            if (tr) atomicAdd(&a.stats->pruned_reach, tr);
        }
    }
}

inline unsigned grid_for(int64_t n, int threads, int64_t cap = 152 * 64) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (unsigned)b;
}

}  // namespace

void ae_children(const ChildrenArgs &a, cudaStream_t st) {
    if (a.nnodes <= 0) return;
    ++g_launches;
    if (a.ix.sigma == 4)
        k_children<4><<<grid_for(a.nnodes, 256), 256, 0, st>>>(a);
    else
        k_children<20><<<grid_for(a.nnodes, 256), 256, 0, st>>>(a);
}

void ae_compact_segs(const ChildrenArgs &a, const uint64_t *seg_off, const uint64_t *trip_off, Seg *segs,
                     uint64_t *task_first, cudaStream_t st) {
    if (a.nnodes <= 0) return;
    ++g_launches;
    if (a.ix.sigma == 4)
        k_compact<4><<<grid_for(a.nnodes, 256), 256, 0, st>>>(a, seg_off, trip_off, segs, task_first);
    else
        k_compact<20><<<grid_for(a.nnodes, 256), 256, 0, st>>>(a, seg_off, trip_off, segs, task_first);
}

template <int SIGMA, bool I16>
void launch_rows(const RowsArgs &a, bool write, int blocks, cudaStream_t st) {
    if (write)
        k_rows<SIGMA, true, I16><<<blocks, RW_WARPS * 32, 0, st>>>(a);
    else
        k_rows<SIGMA, false, I16><<<blocks, RW_WARPS * 32, 0, st>>>(a);
}

int ae_rows_blocks_per_sm(bool write) { return write ? RW_MINB_WRITE : RW_MINB_COUNT; }

void ae_rows(const RowsArgs &a, bool write, int blocks, cudaStream_t st) {
    ++g_launches;
    if (a.ix.sigma == 4) {
        if (a.int16) launch_rows<4, true>(a, write, blocks, st);
        else launch_rows<4, false>(a, write, blocks, st);
    } else {
        if (a.int16) launch_rows<20, true>(a, write, blocks, st);
        else launch_rows<20, false>(a, write, blocks, st);
    }
}

// Leave the int16 route: unpack a level arena of (M | G_a << 16) pairs into
// int32 M (in place) and G_a.
__global__ void k_mg_to_i32(int32_t *M, int32_t *Ga, int64_t n) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t v = reinterpret_cast<const uint32_t *>(M)[t];
        Ga[t] = mg_hi(v);
        M[t] = mg_lo(v);
    }
}

void ae_mg_to_i32(int32_t *M, int32_t *Ga, int64_t n, cudaStream_t st) {
    if (n <= 0) return;
    ++g_launches;
    k_mg_to_i32<<<grid_for(n, 256), 256, 0, st>>>(M, Ga, n);
}
