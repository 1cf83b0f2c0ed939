// Device kernels of exact local-alignment search on sm_103a.
//
// The search walks the suffix trie of T breadth-first through the FM index of
// the reversed text (Section 5): every trie node is an SA range [lo, hi) and
// appending a letter c to its substring is one backward-search step
// (lo' = C[c] + Occ(c, lo), hi' = C[c] + Occ(c, hi)).  Each node carries one
// sparse row of the Gotoh matrix M_X (Section 2.2): the live entries (j, M, G_a)
// sorted by query column j.  A child's row follows from its parent's by the
// three recurrences, where G_b (the in-row horizontal gap) is a max-plus prefix
// scan:  G_b(j) = s_g + j*s_s + max_{k<j} (M'(k) - k*s_s),  M' = max(D, G_a).
// An entry is kept only if its value exceeds
//     thr(j) = max{0, H - 1 - (m - 1 - j) * g_max}          (Theorem 2)
// (the text-length term of Theorem 2 is dropped: keeping more entries is always
// sound).  Starting the walk at depth q-1 from the query's (q-1)-grams is
// Theorem 3; depths beyond L_max (Theorem 1) never hold live entries.
//
// When a child has a single occurrence it leaves the trie: its row becomes an
// "injection" at its text end e.  The sweep kernel then follows such rows
// along the text (the next letter is T[e+1], read from the forward text),
// merging by maximum every row that reaches the same text position: rows of
// different trie paths ending at the same position have the same future, so
// only their per-entry maximum matters.  This is an order-free form of the
// global filter of Theorem 4 (a fork dominated by an alignment that already
// reaches its start cell is not followed separately).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <utility>

#include "ae_device.cuh"
#include "ae_kernels.h"

#define FULL 0xffffffffu

// Kernel launches issued by the calling thread (reported as ae_stats.launches).
thread_local int64_t g_launches = 0;

namespace {
using namespace aedev;

// ------------------------------------------------------------------ scan

constexpr int SC_T = 256, SC_I = 8, SC_TILE = SC_T * SC_I;

template <typename In, int W>
struct InPtrs {
    const In *p[W];
};
template <int W>
struct OutPtrs {
    uint64_t *p[W];
};

template <typename In, int W>
__global__ void __launch_bounds__(SC_T) k_scan_reduce(InPtrs<In, W> in, int64_t N, uint64_t *bsum, int64_t nb) {
    __shared__ uint64_t red[W][SC_T / 32];
    const int64_t base = (int64_t)blockIdx.x * SC_TILE;
    uint64_t s[W];
#pragma unroll
    for (int w = 0; w < W; ++w) s[w] = 0;
    for (int i = 0; i < SC_I; ++i) {
        int64_t idx = base + (int64_t)i * SC_T + threadIdx.x;
        if (idx < N) {
#pragma unroll
            for (int w = 0; w < W; ++w) s[w] += (uint64_t)in.p[w][idx];
        }
    }
#pragma unroll
    for (int w = 0; w < W; ++w) {
        uint64_t v = s[w];
        for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(FULL, v, d);
        if ((threadIdx.x & 31) == 0) red[w][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x < W) {
        uint64_t t = 0;
        for (int k = 0; k < SC_T / 32; ++k) t += red[threadIdx.x][k];
        bsum[(int64_t)threadIdx.x * nb + blockIdx.x] = t;
    }
}

template <typename In, int W>
__global__ void __launch_bounds__(SC_T) k_scan_down(InPtrs<In, W> in, OutPtrs<W> out, int64_t N,
                                                    const uint64_t *boff, int64_t nb, uint64_t *totals) {
    __shared__ uint64_t wsum[W][SC_T / 32];
    const int64_t base = (int64_t)blockIdx.x * SC_TILE + (int64_t)threadIdx.x * SC_I;
    uint64_t v[W][SC_I];
    uint64_t s[W];
#pragma unroll
    for (int w = 0; w < W; ++w) s[w] = 0;
#pragma unroll
    for (int i = 0; i < SC_I; ++i) {
        int64_t idx = base + i;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            v[w][i] = idx < N ? (uint64_t)in.p[w][idx] : 0;
            s[w] += v[w][i];
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint64_t pre[W];
#pragma unroll
    for (int w = 0; w < W; ++w) {
        uint64_t x = s[w];
        for (int d = 1; d < 32; d <<= 1) {
            uint64_t o = __shfl_up_sync(FULL, x, d);
            if (lane >= d) x += o;
        }
        if (lane == 31) wsum[w][wid] = x;
        pre[w] = x - s[w];
    }
    __syncthreads();
#pragma unroll
    for (int w = 0; w < W; ++w) {
        uint64_t add = boff ? boff[(int64_t)w * nb + blockIdx.x] : 0;
        for (int k = 0; k < wid; ++k) add += wsum[w][k];
        uint64_t run = pre[w] + add;
#pragma unroll
        for (int i = 0; i < SC_I; ++i) {
            int64_t idx = base + i;
            if (idx < N) out.p[w][idx] = run;
            run += v[w][i];
        }
        if (totals && blockIdx.x == gridDim.x - 1 && threadIdx.x == SC_T - 1) totals[w] = run;
    }
}

template <typename In, int W>
void scan_rec(const In *const *inp, uint64_t *const *outp, int64_t N, uint64_t *totals, uint64_t *tmp,
              cudaStream_t st) {
    InPtrs<In, W> in;
    OutPtrs<W> out;
    for (int w = 0; w < W; ++w) {
        in.p[w] = inp[w];
        out.p[w] = outp[w];
    }
    if (N <= 0) {
        if (totals) cudaMemsetAsync(totals, 0, sizeof(uint64_t) * W, st);
        return;
    }
    int64_t nb = (N + SC_TILE - 1) / SC_TILE;
    if (nb == 1) {
        ++g_launches;
        k_scan_down<In, W><<<1, SC_T, 0, st>>>(in, out, N, nullptr, 1, totals);
        return;
    }
    uint64_t *bsum = tmp, *boff = tmp + nb * W, *rest = tmp + 2 * nb * W;
    g_launches += 2;
    k_scan_reduce<In, W><<<(unsigned)nb, SC_T, 0, st>>>(in, N, bsum, nb);
    const uint64_t *bin[W];
    uint64_t *bout[W];
    for (int w = 0; w < W; ++w) {
        bin[w] = bsum + w * nb;
        bout[w] = boff + w * nb;
    }
    scan_rec<uint64_t, W>(bin, bout, nb, nullptr, rest, st);
    k_scan_down<In, W><<<(unsigned)nb, SC_T, 0, st>>>(in, out, N, boff, nb, totals);
}

// ------------------------------------------------------------------ radix sort

constexpr int RS_T = 256, RS_TILE = 2048, RS_PER_WARP = 256;

__global__ void __launch_bounds__(RS_T) k_rs_hist(const uint64_t *keys, int64_t N, int shift, uint32_t *hist,
                                                  int64_t ntiles) {
    __shared__ uint32_t cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int i = threadIdx.x; i < RS_TILE; i += RS_T) {
        int64_t idx = base + i;
        if (idx < N) atomicAdd(&cnt[(keys[idx] >> shift) & 255], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

__global__ void __launch_bounds__(RS_T) k_rs_scatter(const uint64_t *kin, const uint32_t *vin, uint64_t *kout,
                                                     uint32_t *vout, int64_t N, int shift, const uint64_t *offs,
                                                     int64_t ntiles) {
    __shared__ uint32_t wcnt[RS_T / 32][256];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int d = lane; d < 256; d += 32) wcnt[wid][d] = 0;
    __syncwarp();
    const int64_t wbase = (int64_t)blockIdx.x * RS_TILE + (int64_t)wid * RS_PER_WARP;
    const unsigned lt = (1u << lane) - 1u;
    for (int r = 0; r < RS_PER_WARP / 32; ++r) {
        int64_t idx = wbase + r * 32 + lane;
        bool valid = idx < N;
        int d = valid ? (int)((kin[idx] >> shift) & 255) : 256;
        unsigned peers = __match_any_sync(FULL, d);
        if (valid && lane == __ffs(peers) - 1) wcnt[wid][d] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    {
        int d = threadIdx.x;
        uint32_t s = 0;
        for (int w = 0; w < RS_T / 32; ++w) {
            uint32_t t = wcnt[w][d];
            wcnt[w][d] = s;
            s += t;
        }
    }
    __syncthreads();
    for (int r = 0; r < RS_PER_WARP / 32; ++r) {
        int64_t idx = wbase + r * 32 + lane;
        bool valid = idx < N;
        uint64_t k = valid ? kin[idx] : 0;
        int d = valid ? (int)((k >> shift) & 255) : 256;
        unsigned peers = __match_any_sync(FULL, d);
        uint32_t basecnt = valid ? wcnt[wid][d] : 0;
        __syncwarp();
        if (valid) {
            int64_t dst = (int64_t)offs[(int64_t)d * ntiles + blockIdx.x] + basecnt + __popc(peers & lt);
            kout[dst] = k;
            vout[dst] = vin[idx];
            if (lane == __ffs(peers) - 1) wcnt[wid][d] = basecnt + __popc(peers);
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------------ queries

__global__ void k_encode(const uint8_t *ascii, uint8_t *codes, int64_t total, int alphabet, int *bad) {
    __shared__ uint8_t lut[256];
    for (int t = threadIdx.x; t < 256; t += blockDim.x) lut[t] = 255;
    __syncthreads();
    if (threadIdx.x == 0) {
        const char *a = alphabet == AE_DNA ? "ACGT" : "ARNDCQEGHILKMFPSTWYV";
        int s = alphabet == AE_DNA ? 4 : 20;
        for (int c = 0; c < s; ++c) lut[(uint8_t)a[c]] = (uint8_t)c;
    }
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint8_t c = lut[ascii[i]];
        if (c == 255) {
            atomicExch(bad, 1);
            c = 0;
        }
        codes[i] = c;
    }
}

// ------------------------------------------------------------------ seed (Theorem 3)

// The part of a seed subtree (its gram) when one search is split over ranks:
// a multiplicative hash spreads neighbouring grams over the parts.
__device__ __forceinline__ int fork_part(uint64_t gram, int parts) {
    return (int)((uint32_t)((gram * 0x9E3779B97F4A7C15ull) >> 32) % (uint32_t)parts);
}

__global__ void k_seed_keys(SeedArgs a, uint64_t *keys, uint32_t *vals) {
    const int bits = a.ix.sigma == 4 ? 2 : 5;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < a.npos;
         t += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = a.nitems;  // largest it with item_pos[it] <= t
        while (hi - lo > 1) {
            int mid = (lo + hi) >> 1;
            if (a.item_pos[mid] <= t) lo = mid; else hi = mid;
        }
        const WorkItem it = a.items[lo];
        const int32_t y = it.c0 + (int32_t)(t - a.item_pos[lo]);
        const uint8_t *P = a.qv.codes + a.qv.off[it.qid];
        uint64_t gram = 0;
        for (int i = 0; i < a.d0; ++i) gram = (gram << bits) | P[y + i];
        keys[t] = ((uint64_t)lo << (bits * a.d0)) | gram;
        vals[t] = (uint32_t)y;
    }
}

__global__ void k_seed_flags(const uint64_t *keys, int64_t N, uint32_t *flags) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N; t += (int64_t)gridDim.x * blockDim.x)
        flags[t] = (t == 0 || keys[t] != keys[t - 1]) ? 1u : 0u;
}

template <int SIGMA>
__global__ void k_seed_nodes(SeedArgs a, const uint64_t *keys, const uint32_t *vals, int64_t N,
                             const uint32_t *flags, const uint64_t *flag_off, Node *nodes, int32_t *aj,
                             int32_t *aM, int32_t *aGa) {
    const int bits = SIGMA == 4 ? 2 : 5;
    const uint64_t gmask = (1ull << (bits * a.d0)) - 1ull;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N; t += (int64_t)gridDim.x * blockDim.x) {
        aj[t] = (int32_t)vals[t] + a.d0 - 1;
        // q-prefix domination (Lemma 1): when every occurrence of the gram in T is
        // preceded by the query letter before its start y, the fork starting at y
        // is matched letter for letter, one better, by the fork starting at y - 1
        // (the same text ends, one more match), so its entry starts dead
        int32_t M0 = a.d0 * a.sc.sa;
        bool dead = false;
        if (a.dom && vals[t] > 0) {
            const WorkItem it = a.items[(int32_t)(keys[t] >> (bits * a.d0))];
            const int prev = a.qv.codes[a.qv.off[it.qid] + vals[t] - 1];
            dead = __ldg(a.dom + (keys[t] & gmask)) == (1u << prev);
        }
        const unsigned dm = __ballot_sync(__activemask(), dead);
        // a search split over ranks keeps the seed subtrees of its own part
        if (a.parts > 1 && fork_part(keys[t] & gmask, a.parts) != a.part) dead = true;
        if (dead && a.dominated && (threadIdx.x & 31) == __ffs(dm) - 1)
            atomicAdd(a.dominated, (unsigned long long)__popc(dm));
        if (dead) M0 = AE_NEG;
        if (a.int16) {
            reinterpret_cast<uint32_t *>(aM)[t] = pack_mg(M0, AE_NEG);
        } else {
            aM[t] = M0;
            aGa[t] = AE_NEG;
        }
        if (flags[t]) {
            uint64_t key = keys[t];
            uint64_t gram = key & gmask;
            uint32_t lo = 0, hi = (uint32_t)a.ix.rows;
            for (int i = a.d0 - 1; i >= 0; --i) {
                int c = (int)((gram >> (bits * i)) & ((1u << bits) - 1u));
                lo = a.ix.C[c] + occ_of<SIGMA>(a.ix, c, lo);
                hi = a.ix.C[c] + occ_of<SIGMA>(a.ix, c, hi);
                if (hi <= lo) { lo = hi = 0; }
            }
            int64_t k = (int64_t)flag_off[t];
            Node nd;
            nd.lo = lo;
            nd.hi = hi;
            nd.item = a.items[(int32_t)(key >> (bits * a.d0))].qid;   // query id, 0 levels unique
            nd.cnt = 0;
            nd.off = (uint64_t)t;
            nodes[k] = nd;
        }
    }
}

// Predecessor masks of the d0-grams of T.  A gram is an occurrence only if it
// lies inside one sequence (collections); its predecessor is the letter before
// it, or `sigma` when it starts a sequence.  Small tables are merged per block
// in shared memory first (the grams of i.i.d. text hit every entry).
__global__ void k_dom_table(IndexView ix, int d0, int bits, uint32_t *mask, int64_t ngram) {
    extern __shared__ uint32_t sm_mask[];
    const bool local = ngram <= 4096;
    if (local) {
        for (int64_t g = threadIdx.x; g < ngram; g += blockDim.x) sm_mask[g] = 0;
        __syncthreads();
    }
    const int64_t last = ix.n - d0;   // last start position
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p <= last; p += (int64_t)gridDim.x * blockDim.x) {
        uint64_t gram = 0;
        bool inside = true;
        for (int i = 0; i < d0; ++i) {
            gram = (gram << bits) | ix.text[p + i];
            if (i + 1 < d0 && seq_end(ix, p + i)) inside = false;
        }
        if (!inside) continue;
        const int prev = (p > 0 && !seq_end(ix, p - 1)) ? (int)ix.text[p - 1] : ix.sigma;
        if (local) atomicOr(&sm_mask[gram], 1u << prev);
        else atomicOr(&mask[gram], 1u << prev);
    }
    if (local) {
        __syncthreads();
        for (int64_t g = threadIdx.x; g < ngram; g += blockDim.x)
            if (sm_mask[g]) atomicOr(&mask[g], sm_mask[g]);
    }
}

__global__ void k_seed_fix(Node *nodes, const uint64_t *nn_dev, int64_t N) {
    const int64_t nn = (int64_t)*nn_dev;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nn; i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t end = (i + 1 < nn) ? nodes[i + 1].off : (uint64_t)N;
        nodes[i].cnt = (uint32_t)(end - nodes[i].off);
    }
}

// ------------------------------------------------------------------ text-position sweep

__global__ void k_inject_keys(const Inject *inj, int64_t ninj, uint64_t *keys, uint32_t *vals) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < ninj; t += (int64_t)gridDim.x * blockDim.x) {
        keys[t] = ((uint64_t)(uint32_t)inj[t].qid << 32) | (uint32_t)inj[t].e;
        vals[t] = (uint32_t)t;
    }
}

struct Buf {
    int32_t *j, *M, *Ga;
};

__device__ __forceinline__ int64_t lower_bound_g(const int32_t *a, int64_t n, int32_t x) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (a[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}
__device__ __forceinline__ int64_t upper_bound_g(const int32_t *a, int64_t n, int32_t x) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (a[mid] <= x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Hit records of the sweep are staged per warp in shared memory and appended
// to the global buffer LEAF_HS at a time, so that the walk along a homologous
// region (hits in most chunks) does not take an atomic on the shared counter
// per chunk.  A chunk with more than LEAF_HS hits reserves global space itself.
constexpr int LEAF_HS = 256;
constexpr int LEAF_WARPS = 4;   // k_leaf runs 128-thread blocks

struct HitStage {
    uint64_t *key;
    int32_t *score;
    uint32_t n;     // staged records (warp-uniform)
    uint32_t cap;   // records the stage holds
};

__device__ __forceinline__ void stage_flush(HitStage &hs, const LeafArgs &a, int lane) {
    __syncwarp();
    if (hs.n == 0) return;
    unsigned long long g = 0;
    if (lane == 0) g = atomicAdd(a.hit_count, (unsigned long long)hs.n);
    g = __shfl_sync(FULL, g, 0);
    if (g + hs.n <= a.hit_cap) {
        for (uint32_t i = lane; i < hs.n; i += 32) {
            a.hit_key[g + i] = hs.key[i];
            a.hit_score[g + i] = hs.score[i];
        }
    } else if (lane == 0) {
        atomicAdd(&a.stats->hit_overflow, 1ull);
    }
    __syncwarp();
    hs.n = 0;
}

// Slots for htot records of this chunk (warp-uniform call): in the stage
// (staged) or in the global buffer (ok = within its capacity).
__device__ __forceinline__ uint64_t stage_reserve(HitStage &hs, const LeafArgs &a, int lane, uint32_t htot,
                                                  bool &staged, bool &ok) {
    if (htot > hs.cap) {
        unsigned long long g = 0;
        if (lane == 0) g = atomicAdd(a.hit_count, (unsigned long long)htot);
        g = __shfl_sync(FULL, g, 0);
        staged = false;
        ok = g + htot <= a.hit_cap;
        if (!ok && lane == 0) atomicAdd(&a.stats->hit_overflow, 1ull);
        return g;
    }
    if (hs.n + htot > hs.cap) stage_flush(hs, a, lane);
    staged = true;
    ok = true;
    const uint64_t b = hs.n;
    hs.n += htot;
    return b;
}

__device__ __forceinline__ void hit_put(HitStage &hs, const LeafArgs &a, bool staged, uint64_t slot, uint64_t key,
                                        int32_t score) {
    if (staged) {
        hs.key[slot] = key;
        hs.score[slot] = score;
    } else {
        a.hit_key[slot] = key;
        a.hit_score[slot] = score;
    }
}

// Slots of one sweep entry (see slot_finish): slot A at the entry's column,
// slot B at the next column unless the next entry is there.
struct Slots {
    int32_t colA, MpA, GaA, MpB, Dp, Dk, next_col;
    bool hasB;
};

__device__ __forceinline__ void make_slots(const ScoreView &sc, const int8_t *smat, int c, const uint8_t *P, int32_t m,
                                           int32_t H, int32_t g, int32_t oe, bool valid, int32_t j, int32_t M,
                                           int32_t Ga, int32_t pj, int32_t pM, int32_t jn, Slots &s) {
    s.colA = m;
    s.MpA = s.GaA = s.MpB = s.Dp = s.Dk = AE_NEG;
    s.next_col = m;
    s.hasB = false;
    if (!valid) return;
    s.colA = j;
    const int32_t tA = thr_of(j, m, H, g);
    if (pj + 1 == j && pM > AE_NEG) {
        const int32_t D = pM + delta_of(sc, smat, c, P[j]);
        s.Dp = D > tA ? D : AE_NEG;
    }
    const int32_t gap = gap_from_i32(M, Ga, sc.ss, oe);
    s.GaA = gap > tA ? gap : AE_NEG;
    s.MpA = max(s.Dp, s.GaA);
    s.hasB = (j + 1 < m) && (j + 1 != jn);
    if (s.hasB) {
        const int32_t D = M + delta_of(sc, smat, c, P[j + 1]);
        s.Dk = D > thr_of(j + 1, m, H, g) ? D : AE_NEG;
        s.MpB = s.Dk;
    }
    s.next_col = jn;
}

// Merge the rows injected at (qid, p) into the walked row Rn (nlen entries).  They are finished rows, and
// the union of two finished rows taken by maximum per column is again
// finished (each is closed under the horizontal-gap recurrence), so the
// merge needs no second finish.  Cells where an injected row brings a
// new or larger value report their hits here.
// Used by the warp walk of k_leaf and, run by one warp, by the block walk of
// k_leaf_wide.
__device__ __forceinline__ void leaf_merge(const LeafArgs &a, int lane, int32_t qid, int32_t p, int32_t H,
                                           uint64_t jmask, int64_t &k, int64_t kend, Buf &Rn, Buf &Cb, Buf &C2,
                                           int64_t &nlen, int64_t cap, bool &overflow, HitStage &hstage,
                                           unsigned long long &st_ent, unsigned long long &st_reused,
                                           unsigned long long &st_t0) {
    while (k < kend) {
        const Inject I = a.inj[a.order[k]];
        if (I.qid != qid || I.e != p) break;
        ++k;
        const int32_t *ij = a.lj + I.off, *iM = a.lM + I.off, *iGa = a.lGa + I.off;
        const int64_t icnt = I.cnt;
        // an injected row whose every entry the walked row already has with
        // M and G_a at least as large changes nothing (its hits were reported
        // with the walked values): skip it.  Along a homologous region the row
        // walked from earlier starts usually dominates the later forks.
        bool dominated = nlen > 0;
        for (int64_t base = 0; dominated && base < icnt; base += 32) {
            const int64_t idx = base + lane;
            bool ok = true;
            if (idx < icnt) {
                const int32_t y = ij[idx];
                const int64_t q = lower_bound_g(Rn.j, nlen, y);
                ok = q < nlen && Rn.j[q] == y && Rn.M[q] >= iM[idx] && Rn.Ga[q] >= iGa[idx];
            }
            dominated = __all_sync(FULL, ok);
        }
        if (dominated) {
            st_reused += (unsigned long long)icnt;   // the whole row rides on the walked one
            continue;
        }
        if (nlen + icnt > cap) {
            overflow = true;
            break;
        }
        for (int64_t base = 0; base < nlen; base += 32) {
            const int64_t idx = base + lane;
            if (idx < nlen) {
                const int32_t x = Rn.j[idx];
                const int64_t d = idx + lower_bound_g(ij, icnt, x);
                C2.j[d] = x;
                C2.M[d] = Rn.M[idx];
                C2.Ga[d] = Rn.Ga[idx];
            }
        }
        for (int64_t base = 0; base < icnt; base += 32) {
            const int64_t idx = base + lane;
            if (idx < icnt) {
                const int32_t y = ij[idx];
                const int64_t d = idx + upper_bound_g(Rn.j, nlen, y);
                C2.j[d] = (int32_t)((uint32_t)y | 0x80000000u);   // tag: from the injected row
                C2.M[d] = iM[idx];
                C2.Ga[d] = iGa[idx];
            }
        }
        __syncwarp();
        // an equal column appears twice: the walked entry first, then the injected one
        const int64_t len2 = nlen + icnt;
        int64_t out = 0;
        const uint64_t kq = ((uint64_t)qid << (a.be + a.bj)) | ((uint64_t)(uint32_t)p << a.bj);
        for (int64_t base = 0; base < len2; base += 32) {
            const int64_t idx = base + lane;
            const bool valid = idx < len2;
            int32_t j = 0, Mv = AE_NEG, Gv = AE_NEG;
            bool keep = false, hit = false, fresh = false;
            if (valid) {
                const uint32_t raw = (uint32_t)C2.j[idx];
                j = (int32_t)(raw & 0x7FFFFFFFu);
                const bool from_inj = raw >> 31;
                Mv = C2.M[idx];
                Gv = C2.Ga[idx];
                keep = !(idx > 0 && (int32_t)((uint32_t)C2.j[idx - 1] & 0x7FFFFFFFu) == j);
                if (keep) {
                    if (idx + 1 < len2 && (int32_t)((uint32_t)C2.j[idx + 1] & 0x7FFFFFFFu) == j) {
                        const int32_t Mi = C2.M[idx + 1];
                        hit = Mi > Mv && Mi >= H;
                        Mv = max(Mv, Mi);
                        Gv = max(Gv, C2.Ga[idx + 1]);
                    } else {
                        fresh = from_inj;
                        hit = from_inj && Mv >= H;
                    }
                }
            }
            const uint32_t ci = warp_incl_sum(keep ? 1u : 0u);
            const uint32_t tot = __shfl_sync(FULL, ci, 31);
            const uint32_t hi = warp_incl_sum(hit ? 1u : 0u);
            const uint32_t htot = __shfl_sync(FULL, hi, 31);
            __syncwarp();
            if (keep) {
                const int64_t d = out + ci - 1;
                Cb.j[d] = j;
                Cb.M[d] = Mv;
                Cb.Ga[d] = Gv;
            }
            if (htot) {
                bool staged, hok;
                const uint64_t hbase = stage_reserve(hstage, a, lane, htot, staged, hok);
                if (hok && hit) hit_put(hstage, a, staged, hbase + hi - 1, kq | ((uint64_t)j & jmask), Mv);
            }
            if (a.tiers && fresh) ++st_t0;
            out += tot;
        }
        __syncwarp();
        st_ent += (unsigned long long)(out - nlen);
        st_reused += (unsigned long long)(nlen + icnt - out);   // columns both rows had
        Buf t = Rn;
        Rn = Cb;
        Cb = t;
        nlen = out;
    }
}

#ifndef AE_LEAF_E
#define AE_LEAF_E 2
#endif
constexpr int LEAF_E = AE_LEAF_E;   // row entries per lane in the wide sweep step

// One warp per segment of `seg` consecutive injections (sorted by query and
// text end).  The warp carries a row R along text positions p, p+1, ...:
//   candidates of row p+1 = the vertical and diagonal slots generated from R
//   with letter T[p+1], merged by maximum with every injected row at p+1;
//   then the horizontal-gap finish of Section 2.2 gives row p+1.
// The walk jumps to the next injection when R has no live entry.  Rows live
// in per-warp global scratch (cap entries per buffer); a row that outgrows it
// sets leaf_overflow and the host reruns with a larger cap.
// A walk whose row grows past esc_min entries is handed on, with the rest of
// its segment, to a slot of k_leaf_wide (a block of threads per walk); when
// the slots are taken the warp carries on itself.  The remaining warp walks
// run fastest with registers to spare: 3 resident blocks per SM (measured).
#ifndef AE_LEAF_MINB
#define AE_LEAF_MINB 3
#endif
__global__ void __launch_bounds__(128, AE_LEAF_MINB) k_leaf(LeafArgs a) {
    __shared__ int8_t smat[AE_MAX_SIGMA * AE_MAX_SIGMA];
    __shared__ uint64_t s_hkey[LEAF_WARPS][LEAF_HS];
    __shared__ int32_t s_hscore[LEAF_WARPS][LEAF_HS];
    load_matrix(a.sc, smat);
    const int lane = threadIdx.x & 31;
    const int gw = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    if (gw >= a.nwarps) return;
    HitStage hstage = {s_hkey[(threadIdx.x >> 5) & (LEAF_WARPS - 1)], s_hscore[(threadIdx.x >> 5) & (LEAF_WARPS - 1)], 0u,
                       (uint32_t)LEAF_HS};
    const ScoreView &sc = a.sc;
    const int32_t u = -sc.ss, oe = sc.sg + sc.ss, g = sc.gmax;
    const int64_t cap = a.cap;
    int32_t *wb = a.scratch + (int64_t)gw * 12 * cap;
    Buf R = {wb, wb + cap, wb + 2 * cap};
    Buf Rn = {wb + 3 * cap, wb + 4 * cap, wb + 5 * cap};
    Buf Cb = {wb + 6 * cap, wb + 7 * cap, wb + 8 * cap};
    Buf C2 = {wb + 9 * cap, wb + 10 * cap, wb + 11 * cap};
    const uint64_t jmask = (1ull << a.bj) - 1ull;
    unsigned long long st_rows = 0, st_ent = 0, st_t0 = 0, st_t1 = 0, st_t2 = 0, st_reused = 0;
    bool overflow = false;

    while (!overflow) {
        unsigned long long s = 0;
        if (lane == 0) s = atomicAdd(a.next_seg, 1ull);
        s = __shfl_sync(FULL, s, 0);
        if (s >= (unsigned long long)a.nseg) break;
        if (*(volatile unsigned long long *)&a.stats->leaf_overflow) break;
        int64_t k = (int64_t)s * a.seg;
        const int64_t kend = min(k + (int64_t)a.seg, a.ninj);
        int64_t rlen = 0;
        int32_t p = -1, qid = -1, m = 0, H = 0;
        const uint8_t *P = nullptr;
        unsigned long long seg_steps = 0, seg_width = 0;
        const long long task_t0 = clock64();
        // R lives in registers (lane i holds entry i) while it has <= 32 entries
        bool inreg = false;
        int32_t rj = 0, rM = AE_NEG, rGa = AE_NEG;
        // text window: lane i holds T[tw_base + i] (one coalesced 32-byte load per
        // 32 positions instead of a dependent random read per step)
        int64_t tw_base = -64;
        uint32_t tw = 0;
        // key (query, text end) of injection k, the next one to merge
        int32_t nk_qid = -1, nk_e = -1;
        if (k < kend) {
            const Inject In = a.inj[a.order[k]];
            nk_qid = In.qid;
            nk_e = In.e;
        }
        while (true) {
            if (rlen == 0 && k < kend) {
                // ---- jump to a lone injected row: it is already a finished row
                const Inject I0 = a.inj[a.order[k]];
                int32_t q2 = -1, e2 = -1;
                if (k + 1 < kend) {
                    const Inject I1 = a.inj[a.order[k + 1]];
                    q2 = I1.qid;
                    e2 = I1.e;
                }
                if (I0.cnt <= 32 && !(q2 == I0.qid && e2 == I0.e)) {
                    p = I0.e;
                    if (I0.qid != qid) {
                        qid = I0.qid;
                        m = a.qv.m[qid];
                        H = a.qv.H[qid];
                        P = a.qv.codes + a.qv.off[qid];
                    }
                    rlen = I0.cnt;
                    if (lane < rlen) {
                        rj = a.lj[I0.off + lane];
                        rM = a.lM[I0.off + lane];
                        rGa = a.lGa[I0.off + lane];
                    }
                    inreg = true;
                    ++k;
                    nk_qid = q2;
                    nk_e = e2;
                    const uint32_t h = (lane < rlen && rM >= H) ? 1u : 0u;
                    const uint32_t hi = warp_incl_sum(h);
                    const uint32_t htot = __shfl_sync(FULL, hi, 31);
                    if (htot) {
                        bool staged, hok;
                        const uint64_t hbase = stage_reserve(hstage, a, lane, htot, staged, hok);
                        if (hok && h) {
                            const uint64_t kq = ((uint64_t)qid << (a.be + a.bj)) | ((uint64_t)(uint32_t)p << a.bj);
                            hit_put(hstage, a, staged, hbase + hi - 1, kq | ((uint64_t)rj & jmask), rM);
                        }
                    }
                    if (a.tiers && lane == 0) st_t0 += (unsigned long long)rlen;   // warp-uniform count
                    ++st_rows;
                    ++seg_steps;
                    st_ent += (unsigned long long)rlen;
                    continue;
                }
            }
            if (rlen > 0 && inreg && p + 1 < a.ix.n && !seq_end(a.ix, p)) {
                const bool inj_next = nk_qid == qid && nk_e == p + 1;
                if (!inj_next) {
                    // ---- fast step: gen + horizontal finish in registers
                    ++p;
                    if (p < tw_base || p >= tw_base + 32) {
                        tw_base = p;
                        tw = (p + lane < a.ix.n) ? a.ix.text[p + lane] : 0u;
                    }
                    const int c = (int)__shfl_sync(FULL, tw, (int)(p - tw_base));
                    const bool valid = lane < rlen;
                    int32_t j = valid ? rj : m, M = valid ? rM : AE_NEG, Ga = valid ? rGa : AE_NEG;
                    int32_t jn = __shfl_down_sync(FULL, j, 1);
                    if (lane + 1 >= rlen) jn = m;
                    int32_t pjv = __shfl_up_sync(FULL, j, 1), pMv = __shfl_up_sync(FULL, M, 1);
                    if (lane == 0) {
                        pjv = -2;
                        pMv = AE_NEG;
                    }
                    int32_t colA = m, MpA = AE_NEG, GaA = AE_NEG, MpB = AE_NEG, next_col = m;
                    int32_t Dp = AE_NEG, Dk = AE_NEG;
                    bool hasB = false;
                    if (valid) {
                        colA = j;
                        const int32_t tA = thr_of(j, m, H, g);
                        if (pjv + 1 == j && pMv > AE_NEG) {
                            const int32_t D = pMv + delta_of(sc, smat, c, P[j]);
                            Dp = D > tA ? D : AE_NEG;
                        }
                        const int32_t gap = gap_from_i32(M, Ga, sc.ss, oe);
                        GaA = gap > tA ? gap : AE_NEG;
                        MpA = max(Dp, GaA);
                        hasB = (j + 1 < m) && (j + 1 != jn);
                        if (hasB) {
                            const int32_t D = M + delta_of(sc, smat, c, P[j + 1]);
                            Dk = D > thr_of(j + 1, m, H, g) ? D : AE_NEG;
                            MpB = Dk;
                        }
                        next_col = jn;
                    }
                    const int32_t keyA = MpA > AE_NEG ? MpA + colA * u : AE_KNEG;
                    const int32_t keyB = MpB > AE_NEG ? MpB + (colA + 1) * u : AE_KNEG;
                    const int32_t incl = warp_incl_max(max(keyA, keyB));
                    int32_t excl = __shfl_up_sync(FULL, incl, 1);
                    if (lane == 0) excl = AE_KNEG;
                    SlotOut o;
                    slot_finish(colA, MpA, hasB, MpB, next_col, excl, incl, sc, m, H, u, valid, o);
                    const uint32_t nA = o.aliveA, nB = o.aliveB, nR = (uint32_t)o.run_len;
                    const uint32_t cn = nA + nB + nR;
                    const uint32_t ci = warp_incl_sum(cn);
                    const uint32_t tot = __shfl_sync(FULL, ci, 31);
                    // hits
                    const uint32_t hA = o.aliveA && o.MA >= H, hB = o.aliveB && o.MB >= H;
                    const uint32_t hc = hA + hB + (uint32_t)o.run_hits;
                    const uint32_t hi = warp_incl_sum(hc);
                    const uint32_t htot = __shfl_sync(FULL, hi, 31);
                    bool staged = true, hok = true;
                    uint64_t hbase = 0;
                    if (htot) hbase = stage_reserve(hstage, a, lane, htot, staged, hok);
                    const uint64_t kq = ((uint64_t)qid << (a.be + a.bj)) | ((uint64_t)(uint32_t)p << a.bj);
                    const uint64_t h0 = hbase + hi - hc;
                    if (hok) {
                        if (hA) hit_put(hstage, a, staged, h0, kq | ((uint64_t)colA & jmask), o.MA);
                        if (hB) hit_put(hstage, a, staged, h0 + hA, kq | ((uint64_t)(colA + 1) & jmask), o.MB);
                    }
                    if (a.tiers) {
                        if (o.aliveA) {
                            const int tier = (Dp > AE_NEG) + (GaA > AE_NEG) + (o.GbA > thr_of(colA, m, H, g));
                            st_t0 += tier <= 1;
                            st_t1 += tier == 2;
                            st_t2 += tier >= 3;
                        }
                        if (o.aliveB) {
                            if ((Dk > AE_NEG) && (o.GbB > thr_of(colA + 1, m, H, g))) ++st_t1; else ++st_t0;
                        }
                        st_t0 += nR;
                    }
                    const int64_t e0 = (int64_t)(ci - cn);
                    if (tot > cap) {
                        overflow = true;
                        break;
                    }
                    // run hits and (for rows wider than a warp) run entries, cooperatively
                    unsigned rmask = __ballot_sync(FULL, nR > 0);
                    const bool spill = tot > 32;
                    while (rmask) {
                        const int L = __ffs(rmask) - 1;
                        rmask &= rmask - 1;
                        const int32_t s0 = __shfl_sync(FULL, o.run_start, L);
                        const int32_t rl = __shfl_sync(FULL, o.run_len, L);
                        const int32_t rh = __shfl_sync(FULL, o.run_hits, L);
                        const int32_t K = __shfl_sync(FULL, incl, L);
                        const int64_t d0 = __shfl_sync(FULL, e0 + nA + nB, L);
                        const uint64_t hd = __shfl_sync(FULL, h0 + hA + hB, L);
                        for (int32_t t = lane; t < rl; t += 32) {
                            const int32_t cc = s0 + t;
                            const int32_t v = sc.sg - cc * u + K;
                            if (spill) {
                                R.j[d0 + t] = cc;
                                R.M[d0 + t] = v;
                                R.Ga[d0 + t] = AE_NEG;
                            }
                            if (t < rh && hok) hit_put(hstage, a, staged, hd + t, kq | ((uint64_t)cc & jmask), v);
                        }
                    }
                    if (spill) {
                        if (o.aliveA) {
                            R.j[e0] = colA;
                            R.M[e0] = o.MA;
                            R.Ga[e0] = GaA;
                        }
                        if (o.aliveB) {
                            R.j[e0 + nA] = colA + 1;
                            R.M[e0 + nA] = o.MB;
                            R.Ga[e0 + nA] = AE_NEG;
                        }
                        inreg = false;
                    } else {
                        // output lane <- the lane whose slots/run produced output number `lane`
                        int s = 0;
#pragma unroll
                        for (int step = 16; step > 0; step >>= 1) {
                            const uint32_t v = __shfl_sync(FULL, ci, s + step - 1);
                            if (v <= (uint32_t)lane) s += step;
                        }
                        const uint32_t ex_s = __shfl_sync(FULL, ci - cn, s);
                        const uint32_t nA_s = __shfl_sync(FULL, nA, s), nB_s = __shfl_sync(FULL, nB, s);
                        const int32_t col_s = __shfl_sync(FULL, colA, s), MA_s = __shfl_sync(FULL, o.MA, s);
                        const int32_t GaA_s = __shfl_sync(FULL, GaA, s), MB_s = __shfl_sync(FULL, o.MB, s);
                        const int32_t rs_s = __shfl_sync(FULL, o.run_start, s), K_s = __shfl_sync(FULL, incl, s);
                        const uint32_t r = (uint32_t)lane - ex_s;
                        if ((uint32_t)lane < tot) {
                            if (r < nA_s) {
                                rj = col_s;
                                rM = MA_s;
                                rGa = GaA_s;
                            } else if (r < nA_s + nB_s) {
                                rj = col_s + 1;
                                rM = MB_s;
                                rGa = AE_NEG;
                            } else {
                                rj = rs_s + (int32_t)(r - nA_s - nB_s);
                                rM = sc.sg - rj * u + K_s;
                                rGa = AE_NEG;
                            }
                        }
                    }
                    __syncwarp();
                    rlen = tot;
                    ++st_rows;
                    ++seg_steps;
                    st_ent += (unsigned long long)tot;
                    continue;
                }
            }
            if (inreg && rlen > 0) {   // the slow path reads R from scratch
                if (lane < rlen) {
                    R.j[lane] = rj;
                    R.M[lane] = rM;
                    R.Ga[lane] = rGa;
                }
                __syncwarp();
            }
            inreg = false;
            int64_t nlen = 0;   // length of the finished row at p, kept in Rn
            if (rlen == 0) {
                // a new walk: the row at p is the union of the rows injected there
                if (k >= kend) break;
                const Inject I0 = a.inj[a.order[k]];
                p = I0.e;
                if (I0.qid != qid) {
                    qid = I0.qid;
                    m = a.qv.m[qid];
                    H = a.qv.H[qid];
                    P = a.qv.codes + a.qv.off[qid];
                }
            } else {
                // the row ends with the text or its sequence: the walk goes on with
                // the next injection
                if (p + 1 >= a.ix.n || seq_end(a.ix, p)) {
                    rlen = 0;
                    continue;
                }
                ++p;
                if (p < tw_base || p >= tw_base + 32) {
                    tw_base = p;
                    tw = (p + lane < a.ix.n) ? a.ix.text[p + lane] : 0u;
                }
                const int c = (int)__shfl_sync(FULL, tw, (int)(p - tw_base));
                // ---- slots from R with letter c and the horizontal finish, straight
                // into Rn (the finished row at p) with its hits.  Each lane takes
                // LEAF_E consecutive entries (a lane-local prefix, then one warp scan
                // per quantity), so a wide row needs LEAF_E times fewer warp steps.
                int32_t carry = AE_KNEG, prev_j = -2, prev_M = AE_NEG;
                // the next chunk's entries are loaded while this chunk is computed
                int32_t nj[LEAF_E], nM[LEAF_E], nG[LEAF_E];
#pragma unroll
                for (int e = 0; e < LEAF_E; ++e) {
                    const int64_t x = (int64_t)lane * LEAF_E + e;
                    const bool v = x < rlen;
                    nj[e] = v ? R.j[x] : m;
                    nM[e] = v ? R.M[x] : AE_NEG;
                    nG[e] = v ? R.Ga[x] : AE_NEG;
                }
                for (int64_t base = 0; base < rlen; base += 32 * LEAF_E) {
                    const int64_t i0 = base + (int64_t)lane * LEAF_E;
                    int32_t jj[LEAF_E], MM[LEAF_E], GG[LEAF_E];
#pragma unroll
                    for (int e = 0; e < LEAF_E; ++e) {
                        jj[e] = nj[e];
                        MM[e] = nM[e];
                        GG[e] = nG[e];
                        const int64_t x = i0 + 32 * LEAF_E + e;
                        const bool v = x < rlen;
                        nj[e] = v ? R.j[x] : m;
                        nM[e] = v ? R.M[x] : AE_NEG;
                        nG[e] = v ? R.Ga[x] : AE_NEG;
                    }
                    // the first entry of the next chunk (lane 0's next load), m past the row
                    int32_t jnext = __shfl_down_sync(FULL, jj[0], 1);
                    const int32_t jfirst_next = __shfl_sync(FULL, nj[0], 0);
                    if (lane == 31) jnext = jfirst_next;
                    int32_t pj0 = __shfl_up_sync(FULL, jj[LEAF_E - 1], 1), pM0 = __shfl_up_sync(FULL, MM[LEAF_E - 1], 1);
                    if (lane == 0) {
                        pj0 = prev_j;
                        pM0 = prev_M;
                    }
                    Slots sl[LEAF_E];
                    int32_t lk[LEAF_E];
#pragma unroll
                    for (int e = 0; e < LEAF_E; ++e) {
                        const bool v = i0 + e < rlen;
                        int32_t jn = (e + 1 < LEAF_E) ? jj[e + 1] : jnext;
                        if (i0 + e + 1 >= rlen) jn = m;
                        const int32_t pj = e ? jj[e - 1] : pj0, pM = e ? MM[e - 1] : pM0;
                        make_slots(sc, smat, c, P, m, H, g, oe, v, jj[e], MM[e], GG[e], pj, pM, jn, sl[e]);
                        const int32_t keyA = sl[e].MpA > AE_NEG ? sl[e].MpA + sl[e].colA * u : AE_KNEG;
                        const int32_t keyB = sl[e].MpB > AE_NEG ? sl[e].MpB + (sl[e].colA + 1) * u : AE_KNEG;
                        lk[e] = max(e ? lk[e - 1] : AE_KNEG, max(keyA, keyB));
                    }
                    int32_t lincl = warp_incl_max(lk[LEAF_E - 1]);
                    int32_t lexcl = __shfl_up_sync(FULL, lincl, 1);
                    if (lane == 0) lexcl = AE_KNEG;
                    lincl = max(lincl, carry);
                    lexcl = max(lexcl, carry);
                    SlotOut o[LEAF_E];
                    int32_t ik[LEAF_E];
                    uint32_t cl = 0, hl = 0;
#pragma unroll
                    for (int e = 0; e < LEAF_E; ++e) {
                        const int32_t ex = e ? max(lexcl, lk[e - 1]) : lexcl;
                        ik[e] = max(lexcl, lk[e]);
                        slot_finish(sl[e].colA, sl[e].MpA, sl[e].hasB, sl[e].MpB, sl[e].next_col, ex, ik[e], sc, m, H,
                                    u, i0 + e < rlen, o[e]);
                        cl += (uint32_t)o[e].aliveA + (uint32_t)o[e].aliveB + (uint32_t)o[e].run_len;
                        hl += (uint32_t)(o[e].aliveA && o[e].MA >= H) + (uint32_t)(o[e].aliveB && o[e].MB >= H) +
                              (uint32_t)o[e].run_hits;
                    }
                    carry = __shfl_sync(FULL, lincl, 31);
                    prev_j = __shfl_sync(FULL, jj[LEAF_E - 1], 31);
                    prev_M = __shfl_sync(FULL, MM[LEAF_E - 1], 31);
                    const uint32_t ci = warp_incl_sum(cl);
                    const uint32_t tot = __shfl_sync(FULL, ci, 31);
                    if (nlen + tot > cap) {
                        overflow = true;
                        break;
                    }
                    const uint32_t hi = warp_incl_sum(hl);
                    const uint32_t htot = __shfl_sync(FULL, hi, 31);
                    bool staged = true, hok = true;
                    uint64_t hbase = 0;
                    if (htot) hbase = stage_reserve(hstage, a, lane, htot, staged, hok);
                    const uint64_t kq = ((uint64_t)qid << (a.be + a.bj)) | ((uint64_t)(uint32_t)p << a.bj);
                    int64_t eo = nlen + (int64_t)(ci - cl);
                    uint64_t ho = hbase + hi - hl;
                    int64_t run_d[LEAF_E];
                    uint64_t run_h[LEAF_E];
#pragma unroll
                    for (int e = 0; e < LEAF_E; ++e) {
                        const uint32_t nA = o[e].aliveA, nB = o[e].aliveB;
                        const uint32_t hA = o[e].aliveA && o[e].MA >= H, hB = o[e].aliveB && o[e].MB >= H;
                        const int32_t colA = sl[e].colA;
                        if (o[e].aliveA) {
                            Rn.j[eo] = colA;
                            Rn.M[eo] = o[e].MA;
                            Rn.Ga[eo] = sl[e].GaA;
                            if (hA && hok) hit_put(hstage, a, staged, ho, kq | ((uint64_t)colA & jmask), o[e].MA);
                            if (a.tiers) {
                                const int tier = (sl[e].Dp > AE_NEG) + (sl[e].GaA > AE_NEG) +
                                                 (o[e].GbA > thr_of(colA, m, H, g));
                                st_t0 += tier <= 1;
                                st_t1 += tier == 2;
                                st_t2 += tier >= 3;
                            }
                        }
                        if (o[e].aliveB) {
                            Rn.j[eo + nA] = colA + 1;
                            Rn.M[eo + nA] = o[e].MB;
                            Rn.Ga[eo + nA] = AE_NEG;
                            if (hB && hok)
                                hit_put(hstage, a, staged, ho + hA, kq | ((uint64_t)(colA + 1) & jmask), o[e].MB);
                            if (a.tiers) {
                                if ((sl[e].Dk > AE_NEG) && (o[e].GbB > thr_of(colA + 1, m, H, g))) ++st_t1; else ++st_t0;
                            }
                        }
                        if (a.tiers) st_t0 += (uint32_t)o[e].run_len;
                        run_d[e] = eo + nA + nB;
                        run_h[e] = ho + hA + hB;
                        eo += nA + nB + (uint32_t)o[e].run_len;
                        ho += hA + hB + (uint32_t)o[e].run_hits;
                    }
#pragma unroll
                    for (int e = 0; e < LEAF_E; ++e) {
                        unsigned rmask = __ballot_sync(FULL, o[e].run_len > 0);
                        while (rmask) {
                            const int L = __ffs(rmask) - 1;
                            rmask &= rmask - 1;
                            const int32_t s0 = __shfl_sync(FULL, o[e].run_start, L);
                            const int32_t rl = __shfl_sync(FULL, o[e].run_len, L);
                            const int32_t rh = __shfl_sync(FULL, o[e].run_hits, L);
                            const int32_t K = __shfl_sync(FULL, ik[e], L);
                            const int64_t d0 = __shfl_sync(FULL, run_d[e], L);
                            const uint64_t hd = __shfl_sync(FULL, run_h[e], L);
                            for (int32_t t = lane; t < rl; t += 32) {
                                const int32_t cc = s0 + t;
                                const int32_t v = sc.sg - cc * u + K;
                                Rn.j[d0 + t] = cc;
                                Rn.M[d0 + t] = v;
                                Rn.Ga[d0 + t] = AE_NEG;
                                if (t < rh && hok) hit_put(hstage, a, staged, hd + t, kq | ((uint64_t)cc & jmask), v);
                            }
                        }
                    }
                    nlen += tot;
                }
                __syncwarp();
                if (overflow) break;
                st_ent += (unsigned long long)nlen;
            }
            leaf_merge(a, lane, qid, p, H, jmask, k, kend, Rn, Cb, C2, nlen, cap, overflow, hstage, st_ent, st_reused,
                       st_t0);
            if (overflow) break;
            if (k < kend) {
                const Inject In = a.inj[a.order[k]];
                nk_qid = In.qid;
                nk_e = In.e;
            } else {
                nk_qid = nk_e = -1;
            }
            Buf t = R;
            R = Rn;
            Rn = t;
            rlen = nlen;
            ++st_rows;
            ++seg_steps;
            seg_width = max(seg_width, (unsigned long long)nlen);
            if (a.esc_min > 0 && rlen > a.esc_min) {
                // a wide row goes on on a whole block (k_leaf_wide), with the rest of
                // this task's injections; the warp takes its next task
                unsigned long long slot = 0;
                if (lane == 0) slot = atomicAdd(a.esc_count, 1ull);
                slot = __shfl_sync(FULL, slot, 0);
                if (slot < (unsigned long long)a.esc_max) {
                    int32_t *eb = a.esc_rows + (int64_t)slot * 12 * cap;
                    for (int64_t i = lane; i < rlen; i += 32) {
                        eb[i] = R.j[i];
                        eb[cap + i] = R.M[i];
                        eb[2 * cap + i] = R.Ga[i];
                    }
                    if (lane == 0) {
                        EscWalk e;
                        e.qid = qid;
                        e.p = p;
                        e.rlen = rlen;
                        e.k = k;
                        e.kend = kend;
                        a.esc[slot] = e;
                    }
                    __syncwarp();
                    rlen = 0;
                    k = kend;
                    continue;
                }
            }
            if (rlen <= 32) {
                if (lane < rlen) {
                    rj = R.j[lane];
                    rM = R.M[lane];
                    rGa = R.Ga[lane];
                }
                inreg = true;
            }
        }
        if (overflow && lane == 0) atomicAdd(&a.stats->leaf_overflow, 1ull);
        if (lane == 0) {
            atomicMax(&a.stats->leaf_max_steps, seg_steps);
            atomicMax(&a.stats->leaf_max_width, seg_width);
            atomicMax(&a.stats->leaf_max_cycles, (unsigned long long)(clock64() - task_t0));
        }
    }
    stage_flush(hstage, a, lane);
    unsigned long long t0 = st_t0, t1 = st_t1, t2 = st_t2;
    for (int d = 16; d > 0; d >>= 1) {
        t0 += __shfl_down_sync(FULL, t0, d);
        t1 += __shfl_down_sync(FULL, t1, d);
        t2 += __shfl_down_sync(FULL, t2, d);
    }
    if (lane == 0) {
        if (st_rows) atomicAdd(&a.stats->leaf_rows, st_rows);
        if (st_ent) {
            atomicAdd(&a.stats->entries, st_ent);
            atomicAdd(&a.stats->entries_leaf, st_ent);
        }
        if (t0) atomicAdd(&a.stats->tier[0], t0);
        if (t1) atomicAdd(&a.stats->tier[1], t1);
        if (t2) atomicAdd(&a.stats->tier[2], t2);
        if (st_reused) atomicAdd(&a.stats->reused, st_reused);
    }
}

// ------------------------------------------------------------------ wide sweep walks
//
// A walk whose row has grown wide is continued by a whole block: each step's
// entries are spread over LEAF_WIDE_THREADS threads (LEAF_E consecutive
// entries each), the horizontal-gap keys and the output counts are block-wide
// scans, and the merges of injected rows run on the first warp.  The values
// are those of the warp walk of k_leaf (the same make_slots / slot_finish per
// entry, the same merge); only the time per step differs.
constexpr int LEAF_WIDE_THREADS = 512;
constexpr int LEAF_WIDE_WARPS = LEAF_WIDE_THREADS / 32;
constexpr int LEAF_WIDE_HS = 128;   // hit records staged per warp of the block

__device__ __forceinline__ int32_t block_excl_max(int32_t v, int32_t *sw, int32_t &total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int32_t incl = warp_incl_max(v);
    if (lane == 31) sw[w] = incl;
    __syncthreads();
    int32_t pre = AE_KNEG, all = AE_KNEG;
#pragma unroll
    for (int x = 0; x < LEAF_WIDE_WARPS; ++x) {
        const int32_t y = sw[x];
        if (x < w) pre = max(pre, y);
        all = max(all, y);
    }
    int32_t ex = __shfl_up_sync(FULL, incl, 1);
    if (lane == 0) ex = AE_KNEG;
    total = all;
    __syncthreads();
    return max(pre, ex);
}

__device__ __forceinline__ uint32_t block_excl_sum(uint32_t v, uint32_t *sw, uint32_t &total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t incl = warp_incl_sum(v);
    if (lane == 31) sw[w] = incl;
    __syncthreads();
    uint32_t pre = 0, all = 0;
#pragma unroll
    for (int x = 0; x < LEAF_WIDE_WARPS; ++x) {
        const uint32_t y = sw[x];
        if (x < w) pre += y;
        all += y;
    }
    total = all;
    __syncthreads();
    return pre + incl - v;
}

struct WideState {
    int64_t rlen, k;
    int32_t p, qid, m, H;
    int32_t buf[4];   // the slot's buffers serving as R, Rn, Cb, C2
    int32_t overflow;
};

__global__ void __launch_bounds__(LEAF_WIDE_THREADS) k_leaf_wide(LeafArgs a) {
    __shared__ int8_t smat[AE_MAX_SIGMA * AE_MAX_SIGMA];
    __shared__ uint64_t s_hkey[LEAF_WIDE_WARPS][LEAF_WIDE_HS];
    __shared__ int32_t s_hscore[LEAF_WIDE_WARPS][LEAF_WIDE_HS];
    __shared__ uint32_t s_scan[LEAF_WIDE_WARPS];
    __shared__ WideState ws;
    load_matrix(a.sc, smat);
    const unsigned long long nesc = min(*(volatile unsigned long long *)a.esc_count, (unsigned long long)a.esc_max);
    if ((unsigned long long)blockIdx.x >= nesc) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    HitStage hstage = {s_hkey[wid], s_hscore[wid], 0u, (uint32_t)LEAF_WIDE_HS};
    const ScoreView &sc = a.sc;
    const int32_t u = -sc.ss, oe = sc.sg + sc.ss, g = sc.gmax;
    const int64_t cap = a.cap;
    const uint64_t jmask = (1ull << a.bj) - 1ull;
    int32_t *eb = a.esc_rows + (int64_t)blockIdx.x * 12 * cap;
    Buf B[4];
#pragma unroll
    for (int x = 0; x < 4; ++x) B[x] = Buf{eb + 3 * x * cap, eb + (3 * x + 1) * cap, eb + (3 * x + 2) * cap};
    const EscWalk e0 = a.esc[blockIdx.x];
    const int64_t kend = e0.kend;
    if (threadIdx.x == 0) {
        ws.rlen = e0.rlen;
        ws.k = e0.k;
        ws.p = e0.p;
        ws.qid = e0.qid;
        ws.m = a.qv.m[e0.qid];
        ws.H = a.qv.H[e0.qid];
        for (int x = 0; x < 4; ++x) ws.buf[x] = x;
        ws.overflow = 0;
    }
    __syncthreads();
    unsigned long long st_rows = 0, st_ent = 0, st_reused = 0, st_t0 = 0, steps = 0, width = 0;
    const long long t_start = clock64();
    while (true) {
        const int64_t rlen = ws.rlen;
        int64_t k = ws.k;
        int32_t p = ws.p, qid = ws.qid, m = ws.m, H = ws.H;
        const int ib[4] = {ws.buf[0], ws.buf[1], ws.buf[2], ws.buf[3]};
        __syncthreads();   // every thread has the state before thread 0 changes it
        Buf R = B[ib[0]], Rn = B[ib[1]], Cb = B[ib[2]], C2 = B[ib[3]];
        int64_t nlen = 0;
        if (rlen == 0) {
            if (k >= kend) break;
            // a new walk: the row at p is the union of the rows injected there
            const Inject I0 = a.inj[a.order[k]];
            p = I0.e;
            qid = I0.qid;
            m = a.qv.m[qid];
            H = a.qv.H[qid];
        } else {
            if (p + 1 >= a.ix.n || seq_end(a.ix, p)) {   // the walk ends with the text or its sequence
                if (threadIdx.x == 0) ws.rlen = 0;
                __syncthreads();
                continue;
            }
            ++p;
            const int c = (int)a.ix.text[p];
            const uint8_t *P = a.qv.codes + a.qv.off[qid];
            int32_t carry = AE_KNEG;
            bool ovf = false;
            for (int64_t base = 0; base < rlen; base += (int64_t)LEAF_WIDE_THREADS * LEAF_E) {
                const int64_t i0 = base + (int64_t)threadIdx.x * LEAF_E;
                int32_t jj[LEAF_E], MM[LEAF_E], GG[LEAF_E];
#pragma unroll
                for (int e = 0; e < LEAF_E; ++e) {
                    const bool v = i0 + e < rlen;
                    jj[e] = v ? R.j[i0 + e] : m;
                    MM[e] = v ? R.M[i0 + e] : AE_NEG;
                    GG[e] = v ? R.Ga[i0 + e] : AE_NEG;
                }
                // the entries around this thread's: the next one's column, the previous one
                const int32_t jnext = i0 + LEAF_E < rlen ? R.j[i0 + LEAF_E] : m;
                int32_t pj0 = -2, pM0 = AE_NEG;
                if (i0 > 0 && i0 - 1 < rlen) {
                    pj0 = R.j[i0 - 1];
                    pM0 = R.M[i0 - 1];
                }
                Slots sl[LEAF_E];
                int32_t lk[LEAF_E];
#pragma unroll
                for (int e = 0; e < LEAF_E; ++e) {
                    const bool v = i0 + e < rlen;
                    int32_t jn = (e + 1 < LEAF_E) ? jj[e + 1] : jnext;
                    if (i0 + e + 1 >= rlen) jn = m;
                    const int32_t pj = e ? jj[e - 1] : pj0, pM = e ? MM[e - 1] : pM0;
                    make_slots(sc, smat, c, P, m, H, g, oe, v, jj[e], MM[e], GG[e], pj, pM, jn, sl[e]);
                    const int32_t keyA = sl[e].MpA > AE_NEG ? sl[e].MpA + sl[e].colA * u : AE_KNEG;
                    const int32_t keyB = sl[e].MpB > AE_NEG ? sl[e].MpB + (sl[e].colA + 1) * u : AE_KNEG;
                    lk[e] = max(e ? lk[e - 1] : AE_KNEG, max(keyA, keyB));
                }
                int32_t kall;
                int32_t lexcl = block_excl_max(lk[LEAF_E - 1], (int32_t *)s_scan, kall);
                lexcl = max(lexcl, carry);
                carry = max(carry, kall);
                SlotOut o[LEAF_E];
                uint32_t cl = 0, hl = 0;
                int32_t ik[LEAF_E];
#pragma unroll
                for (int e = 0; e < LEAF_E; ++e) {
                    const int32_t ex = e ? max(lexcl, lk[e - 1]) : lexcl;
                    ik[e] = max(lexcl, lk[e]);
                    slot_finish(sl[e].colA, sl[e].MpA, sl[e].hasB, sl[e].MpB, sl[e].next_col, ex, ik[e], sc, m, H, u,
                                i0 + e < rlen, o[e]);
                    cl += (uint32_t)o[e].aliveA + (uint32_t)o[e].aliveB + (uint32_t)o[e].run_len;
                    hl += (uint32_t)(o[e].aliveA && o[e].MA >= H) + (uint32_t)(o[e].aliveB && o[e].MB >= H) +
                          (uint32_t)o[e].run_hits;
                }
                uint32_t ctot;
                const uint32_t cex = block_excl_sum(cl, s_scan, ctot);
                if (nlen + (int64_t)ctot > cap) {   // block-uniform
                    ovf = true;
                    break;
                }
                // hits: each warp reserves its own in its stage
                const uint32_t hi = warp_incl_sum(hl);
                const uint32_t htot = __shfl_sync(FULL, hi, 31);
                bool staged = true, hok = true;
                uint64_t hbase = 0;
                if (htot) hbase = stage_reserve(hstage, a, lane, htot, staged, hok);
                const uint64_t kq = ((uint64_t)qid << (a.be + a.bj)) | ((uint64_t)(uint32_t)p << a.bj);
                int64_t eo = nlen + (int64_t)cex;
                uint64_t ho = hbase + hi - hl;
#pragma unroll
                for (int e = 0; e < LEAF_E; ++e) {
                    const int32_t colA = sl[e].colA;
                    const bool hA = o[e].aliveA && o[e].MA >= H, hB = o[e].aliveB && o[e].MB >= H;
                    if (o[e].aliveA) {
                        Rn.j[eo] = colA;
                        Rn.M[eo] = o[e].MA;
                        Rn.Ga[eo] = sl[e].GaA;
                        ++eo;
                        if (hA && hok) hit_put(hstage, a, staged, ho, kq | ((uint64_t)colA & jmask), o[e].MA);
                        ho += hA;
                    }
                    if (o[e].aliveB) {
                        Rn.j[eo] = colA + 1;
                        Rn.M[eo] = o[e].MB;
                        Rn.Ga[eo] = AE_NEG;
                        ++eo;
                        if (hB && hok) hit_put(hstage, a, staged, ho, kq | ((uint64_t)(colA + 1) & jmask), o[e].MB);
                        ho += hB;
                    }
                    for (int32_t r = 0; r < o[e].run_len; ++r) {
                        const int32_t cc = o[e].run_start + r;
                        const int32_t v = sc.sg - cc * u + ik[e];
                        Rn.j[eo] = cc;
                        Rn.M[eo] = v;
                        Rn.Ga[eo] = AE_NEG;
                        ++eo;
                        if (r < o[e].run_hits) {
                            if (hok) hit_put(hstage, a, staged, ho, kq | ((uint64_t)cc & jmask), v);
                            ++ho;
                        }
                    }
                }
                nlen += (int64_t)ctot;
            }
            if (ovf) {
                if (threadIdx.x == 0) ws.overflow = 1;
                __syncthreads();
                break;
            }
            st_ent += (unsigned long long)nlen;
            __syncthreads();   // the step's row is complete before the merge reads it
        }
        // ---- the rows injected at (qid, p), merged by the first warp
        if (wid == 0) {
            bool ovf = false;
            leaf_merge(a, lane, qid, p, H, jmask, k, kend, Rn, Cb, C2, nlen, cap, ovf, hstage, st_ent, st_reused,
                       st_t0);
            if (lane == 0) {
                int nr = ib[1], nc = ib[2];   // the merge may have exchanged Rn and Cb
                if (Rn.j != B[ib[1]].j) {
                    nr = ib[2];
                    nc = ib[1];
                }
                ws.buf[0] = nr;   // the finished row at p
                ws.buf[1] = ib[0];
                ws.buf[2] = nc;
                ws.buf[3] = ib[3];
                ws.rlen = nlen;
                ws.k = k;
                ws.p = p;
                ws.qid = qid;
                ws.m = m;
                ws.H = H;
                if (ovf) ws.overflow = 1;
            }
        }
        __syncthreads();
        if (ws.overflow) break;
        ++st_rows;
        ++steps;
        width = max(width, (unsigned long long)ws.rlen);
    }
    stage_flush(hstage, a, lane);
    if (threadIdx.x == 0) {
        if (ws.overflow) atomicAdd(&a.stats->leaf_overflow, 1ull);
        if (st_rows) atomicAdd(&a.stats->leaf_rows, st_rows);
        if (st_ent) {
            atomicAdd(&a.stats->entries, st_ent);
            atomicAdd(&a.stats->entries_leaf, st_ent);
        }
        if (st_reused) atomicAdd(&a.stats->reused, st_reused);
        atomicMax(&a.stats->leaf_max_steps, steps);
        atomicMax(&a.stats->leaf_max_width, width);
        atomicMax(&a.stats->leaf_max_cycles, (unsigned long long)(clock64() - t_start));
    }
}

// ------------------------------------------------------------------ locate + reduce

__global__ void k_locate_counts(const RangeHit *rh, int64_t n, uint32_t *cnt) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        cnt[t] = rh[t].hi - rh[t].lo;
}

__global__ void k_locate(const RangeHit *rh, int64_t n, const uint64_t *off, int64_t total, const int32_t *tend,
                         int be, int bj, uint64_t *key, int32_t *score) {
    const uint64_t jmask = (1ull << bj) - 1ull;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = n;  // largest r with off[r] <= t
        while (hi - lo > 1) {
            int64_t mid = (lo + hi) >> 1;
            if ((int64_t)off[mid] <= t) lo = mid; else hi = mid;
        }
        const RangeHit r = rh[lo];
        const int64_t row = r.lo + (t - (int64_t)off[lo]);
        const int32_t e = tend[row];
        key[t] = ((uint64_t)(uint32_t)r.qid << (be + bj)) | ((uint64_t)(uint32_t)e << bj) | ((uint64_t)r.j & jmask);
        score[t] = r.score;
    }
}

// Keys (query, text end, query end) of result records to merge, their scores as values.
__global__ void k_merge_keys(const ae_hit *hits, const int32_t *qid, int64_t N, int be, int bj, uint64_t *key,
                             uint32_t *val) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N; t += (int64_t)gridDim.x * blockDim.x) {
        const ae_hit h = hits[t];
        key[t] = ((uint64_t)(uint32_t)qid[t] << (be + bj)) | ((uint64_t)h.text_end << bj) | (uint64_t)(uint32_t)h.query_end;
        val[t] = (uint32_t)h.score;
    }
}

__global__ void k_unique_flags(const uint64_t *key, int64_t N, uint32_t *flags) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N; t += (int64_t)gridDim.x * blockDim.x)
        flags[t] = (t == 0 || key[t] != key[t - 1]) ? 1u : 0u;
}

__global__ void k_unique_write(const uint64_t *key, const int32_t *score, int64_t N, const uint64_t *off, int be,
                               int bj, ae_hit *out, unsigned long long *qcount) {
    const uint64_t jmask = (1ull << bj) - 1ull, emask = (1ull << be) - 1ull;
    const int lane = threadIdx.x & 31;
    // the loop bound is uniform over a warp, so every lane reaches the per-query vote
    for (int64_t t0 = blockIdx.x * (int64_t)blockDim.x; t0 < N; t0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = t0 + threadIdx.x;
        uint32_t q = 0xFFFFFFFFu;   // the query of a cell's first record, else none
        if (t < N) {
            const uint64_t k = key[t];
            if (!(t > 0 && key[t - 1] == k)) {
                int32_t best = score[t];
                for (int64_t u = t + 1; u < N && key[u] == k; ++u) best = max(best, score[u]);
                ae_hit h;
                h.text_end = (int64_t)((k >> bj) & emask);
                h.query_end = (int32_t)(k & jmask);
                h.score = best;
                out[off ? off[t] : t] = h;   // off NULL: the records are unique already
                q = (uint32_t)(k >> (be + bj));
            }
        }
        // per-query counts: one atomic per query present in the warp (the records are
        // sorted by query, so a warp usually holds one or two)
        const unsigned grp = __match_any_sync(FULL, q);
        if (q != 0xFFFFFFFFu && lane == __ffs(grp) - 1) atomicAdd(&qcount[q], (unsigned long long)__popc(grp));
    }
}

__global__ void k_unique_compact(const uint64_t *key, const int32_t *score, int64_t N, const uint64_t *off,
                                 uint64_t *okey, int32_t *oscore) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N; t += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = key[t];
        if (t > 0 && key[t - 1] == k) continue;
        int32_t best = score[t];
        for (int64_t u = t + 1; u < N && key[u] == k; ++u) best = max(best, score[u]);
        okey[off[t]] = k;
        oscore[off[t]] = best;
    }
}

inline unsigned grid_for(int64_t n, int threads, int64_t cap = 152 * 64) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (unsigned)b;
}

}  // namespace

// ------------------------------------------------------------------ launch wrappers

int64_t ae_launches_read() { return g_launches; }


int64_t ae_scan_tmp_words(int64_t N, int W) {
    int64_t words = 0;
    while (N > SC_TILE) {
        int64_t nb = (N + SC_TILE - 1) / SC_TILE;
        words += 2 * nb * W;
        N = nb;
    }
    return words + 8;
}

void ae_scan_u32(const uint32_t *const *in, uint64_t *const *out, int W, int64_t N, uint64_t *totals,
                 uint64_t *tmp, cudaStream_t st) {
    switch (W) {
        case 1: scan_rec<uint32_t, 1>(in, out, N, totals, tmp, st); break;
        case 2: scan_rec<uint32_t, 2>(in, out, N, totals, tmp, st); break;
        case 5: scan_rec<uint32_t, 5>(in, out, N, totals, tmp, st); break;
        default: break;
    }
}

int64_t ae_sort_tmp_words(int64_t N) {
    int64_t ntiles = (N + RS_TILE - 1) / RS_TILE;
    int64_t h = 256 * ntiles;
    // hist (u32, packed two per word) + offsets (u64) + scan tmp
    return (h + 1) / 2 + h + ae_scan_tmp_words(h, 1) + 8;
}

int ae_radix_sort(uint64_t *k0, uint32_t *v0, uint64_t *k1, uint32_t *v1, int64_t N, int bits, uint64_t *tmp,
                  cudaStream_t st) {
    if (N <= 1 || bits <= 0) return 0;
    const int64_t ntiles = (N + RS_TILE - 1) / RS_TILE;
    const int64_t h = 256 * ntiles;
    uint32_t *hist = reinterpret_cast<uint32_t *>(tmp);
    uint64_t *offs = tmp + (h + 1) / 2;
    uint64_t *stmp = offs + h;
    int which = 0;
    for (int shift = 0; shift < bits; shift += 8) {
        uint64_t *ki = which ? k1 : k0, *ko = which ? k0 : k1;
        uint32_t *vi = which ? v1 : v0, *vo = which ? v0 : v1;
        ++g_launches;
        k_rs_hist<<<(unsigned)ntiles, RS_T, 0, st>>>(ki, N, shift, hist, ntiles);
        const uint32_t *in[1] = {hist};
        uint64_t *out[1] = {offs};
        scan_rec<uint32_t, 1>(in, out, h, nullptr, stmp, st);
        ++g_launches;
        k_rs_scatter<<<(unsigned)ntiles, RS_T, 0, st>>>(ki, vi, ko, vo, N, shift, offs, ntiles);
        which ^= 1;
    }
    return which;
}

void ae_encode_queries(const uint8_t *ascii, uint8_t *codes, int64_t total, int alphabet, int *bad,
                       cudaStream_t st) {
    if (total <= 0) return;
    ++g_launches;
    k_encode<<<grid_for(total, 256), 256, 0, st>>>(ascii, codes, total, alphabet, bad);
}

void ae_seed_keys(const SeedArgs &a, uint64_t *keys, uint32_t *vals, cudaStream_t st) {
    if (a.npos <= 0) return;
    ++g_launches;
    k_seed_keys<<<grid_for(a.npos, 256), 256, 0, st>>>(a, keys, vals);
}

void ae_seed_nodes(const SeedArgs &a, const uint64_t *keys, const uint32_t *vals, int64_t npos, int key_bits,
                   uint32_t *flags, uint64_t *flag_off, uint64_t *tmp, Node *nodes, int32_t *aj, int32_t *aM,
                   int32_t *aGa, uint64_t *nnodes_dev, cudaStream_t st) {
    (void)key_bits;
    if (npos <= 0) {
        cudaMemsetAsync(nnodes_dev, 0, sizeof(uint64_t), st);
        return;
    }
    ++g_launches;
    k_seed_flags<<<grid_for(npos, 256), 256, 0, st>>>(keys, npos, flags);
    const uint32_t *in[1] = {flags};
    uint64_t *out[1] = {flag_off};
    scan_rec<uint32_t, 1>(in, out, npos, nnodes_dev, tmp, st);
    ++g_launches;
    if (a.ix.sigma == 4)
        k_seed_nodes<4><<<grid_for(npos, 256), 256, 0, st>>>(a, keys, vals, npos, flags, flag_off, nodes, aj, aM, aGa);
    else
        k_seed_nodes<20><<<grid_for(npos, 256), 256, 0, st>>>(a, keys, vals, npos, flags, flag_off, nodes, aj, aM, aGa);
    ++g_launches;
    k_seed_fix<<<grid_for(npos, 256), 256, 0, st>>>(nodes, nnodes_dev, npos);
}

void ae_dom_table(const IndexView &ix, int d0, uint32_t *mask, cudaStream_t st) {
    const int bits = ix.sigma == 4 ? 2 : 5;
    const int64_t ngram = 1ll << (bits * d0);
    if (ix.n < d0) return;
    ++g_launches;
    const size_t smem = ngram <= 4096 ? (size_t)ngram * 4 : 0;
    k_dom_table<<<grid_for(ix.n, 256, 152 * 8), 256, smem, st>>>(ix, d0, bits, mask, ngram);
}

void ae_inject_keys(const Inject *inj, int64_t ninj, uint64_t *keys, uint32_t *vals, cudaStream_t st) {
    if (ninj <= 0) return;
    ++g_launches;
    k_inject_keys<<<grid_for(ninj, 256), 256, 0, st>>>(inj, ninj, keys, vals);
}

int64_t ae_leaf_scratch_words(int32_t cap, int32_t nwarps) { return (int64_t)12 * cap * nwarps; }

void ae_leaf_sweep(const LeafArgs &a, int blocks, int threads, cudaStream_t st) {
    if (a.nseg <= 0) return;
    ++g_launches;
    k_leaf<<<blocks, threads, 0, st>>>(a);
    if (a.esc_min > 0 && a.esc_max > 0) {   // the walks handed on to blocks (a block per slot taken)
        ++g_launches;
        k_leaf_wide<<<a.esc_max, LEAF_WIDE_THREADS, 0, st>>>(a);
    }
}

void ae_locate_counts(const RangeHit *rh, int64_t nrh, uint32_t *cnt, cudaStream_t st) {
    if (nrh <= 0) return;
    ++g_launches;
    k_locate_counts<<<grid_for(nrh, 256), 256, 0, st>>>(rh, nrh, cnt);
}

void ae_locate(const RangeHit *rh, int64_t nrh, const uint64_t *off, int64_t total, const int32_t *tend, int be,
                 int bj, uint64_t *key, int32_t *score, cudaStream_t st) {
    if (total <= 0) return;
    ++g_launches;
    k_locate<<<grid_for(total, 256), 256, 0, st>>>(rh, nrh, off, total, tend, be, bj, key, score);
}

void ae_merge_keys(const ae_hit *hits, const int32_t *qid, int64_t N, int be, int bj, uint64_t *key, uint32_t *val,
                   cudaStream_t st) {
    if (N <= 0) return;
    ++g_launches;
    k_merge_keys<<<grid_for(N, 256), 256, 0, st>>>(hits, qid, N, be, bj, key, val);
}

void ae_unique_flags(const uint64_t *key, int64_t N, uint32_t *flags, cudaStream_t st) {
    if (N <= 0) return;
    ++g_launches;
    k_unique_flags<<<grid_for(N, 256), 256, 0, st>>>(key, N, flags);
}

void ae_unique_compact(const uint64_t *key, const int32_t *score, int64_t N, const uint64_t *flag_off, uint64_t *okey,
                       int32_t *oscore, cudaStream_t st) {
    if (N <= 0) return;
    ++g_launches;
    k_unique_compact<<<grid_for(N, 256), 256, 0, st>>>(key, score, N, flag_off, okey, oscore);
}

void ae_unique_write(const uint64_t *key, const int32_t *score, int64_t N, const uint64_t *flag_off, int be, int bj,
                     ae_hit *out, unsigned long long *qcount, cudaStream_t st) {
    if (N <= 0) return;
    ++g_launches;
    k_unique_write<<<grid_for(N, 256), 256, 0, st>>>(key, score, N, flag_off, be, bj, out, qcount);
}

// ------------------------------------------------------------------ suffix array by prefix doubling
//
// The suffix array of Section 2.3 (Section 5 (1) builds it over the reversed
// text), computed on the device by prefix doubling (Manber & Myers, 1993):
// every suffix gets a key that orders it by its first h letters, a stable
// radix sort groups equal keys, the group index becomes the suffix's rank,
// and the next key is the pair (rank of the suffix, rank of the suffix h
// letters on), which orders by the first 2h letters.  Rounds stop when every
// rank is distinct.  The first key packs the first 64 / b letters directly
// (b bits per letter value, the sentinel 0 included), so an i.i.d. text of
// 10^8 letters needs one pair round.

namespace {

// s[k] = letter + 1 of the text (read backwards with `reversed`), s[n] = 0
__global__ void k_sa_letters(const uint8_t *codes, int64_t n, int reversed, int sigma, uint8_t *s, int *bad) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k <= n; k += (int64_t)gridDim.x * blockDim.x) {
        uint8_t v = 0;
        if (k < n) {
            const uint8_t c = codes[reversed ? n - 1 - k : k];
            if (c >= sigma) *bad = 1;
            v = (uint8_t)(c + 1);
        }
        s[k] = v;
    }
}

// key of suffix i: its first L letter values, b bits each, first letter highest;
// positions past the sentinel read 0 (the sentinel is unique, so this never ties
// two different suffixes)
__global__ void k_sa_first_keys(const uint8_t *s, int64_t N, int b, int L, uint64_t *keys, uint32_t *vals) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t key = 0;
        for (int t = 0; t < L; ++t) {
            const int64_t x = i + t;
            key = (key << b) | (uint64_t)(x < N ? s[x] : 0);
        }
        keys[i] = key;
        vals[i] = (uint32_t)i;
    }
}

// 1 where a sorted key starts a new group
__global__ void k_sa_heads(const uint64_t *keys, int64_t N, uint32_t *head) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x)
        head[p] = (p == 0 || keys[p] != keys[p - 1]) ? 1u : 0u;
}

// rank of suffix vals[p] = index of its group (inclusive count of heads - 1)
__global__ void k_sa_rank(const uint32_t *vals, const uint32_t *head, const uint64_t *excl, int64_t N,
                          uint32_t *rank, int *bad) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t i = vals[p];
        if ((int64_t)i >= N) {
            *bad = 2;
            continue;
        }
        rank[i] = (uint32_t)(excl[p] + head[p] - 1);
    }
}

// key of suffix i for the 2h-letter order: (rank of i, rank of i + h plus one);
// a suffix shorter than h + 1 letters holds the sentinel in its first h letters,
// so its rank is already unique and its second component is 0
__global__ void k_sa_pair_keys(const uint32_t *rank, int64_t N, int64_t h, int rb, uint64_t *keys, uint32_t *vals) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t second = (i + h < N) ? (uint64_t)rank[i + h] + 1u : 0u;
        keys[i] = ((uint64_t)rank[i] << rb) | second;
        vals[i] = (uint32_t)i;
    }
}

int sa_bits_for(uint64_t maxval) {  // bits to hold values in [0, maxval]
    int b = 1;
    while (b < 64 && (maxval >> b) != 0) ++b;
    return b;
}

}  // namespace

ae_status ae_sa_doubling(const uint8_t *d_codes, int64_t n, int sigma, int reversed, int32_t *d_sa, int *rounds,
                         cudaStream_t st) {
    const int64_t N = n + 1;
    if (rounds) *rounds = 0;
    const int b = sa_bits_for((uint64_t)sigma), L = 64 / b;
    uint8_t *s = nullptr;
    uint64_t *k0 = nullptr, *k1 = nullptr, *tmp = nullptr, *total = nullptr;
    uint32_t *v0 = nullptr, *v1 = nullptr, *rank = nullptr;
    int *bad = nullptr;
    const int64_t tmp_words = std::max(ae_sort_tmp_words(N), ae_scan_tmp_words(N, 1));
    ae_status res = AE_OK;
    if (cudaMalloc(&s, (size_t)N) != cudaSuccess || cudaMalloc(&k0, sizeof(uint64_t) * N) != cudaSuccess ||
        cudaMalloc(&k1, sizeof(uint64_t) * N) != cudaSuccess || cudaMalloc(&v0, sizeof(uint32_t) * N) != cudaSuccess ||
        cudaMalloc(&v1, sizeof(uint32_t) * N) != cudaSuccess ||
        cudaMalloc(&rank, sizeof(uint32_t) * N) != cudaSuccess ||
        cudaMalloc(&tmp, sizeof(uint64_t) * tmp_words) != cudaSuccess ||
        cudaMalloc(&total, sizeof(uint64_t)) != cudaSuccess || cudaMalloc(&bad, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        res = AE_ENOMEM;
    }
    int h_bad = 0;
    uint64_t G = 0;
    if (res == AE_OK && cudaMemsetAsync(bad, 0, sizeof(int), st) != cudaSuccess) res = AE_ECUDA;
    if (res == AE_OK) {
        g_launches += 2;
        k_sa_letters<<<grid_for(N, 256), 256, 0, st>>>(d_codes, n, reversed, sigma, s, bad);
        k_sa_first_keys<<<grid_for(N, 256), 256, 0, st>>>(s, N, b, L, k0, v0);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            res = AE_ECUDA;
        else if (h_bad)
            res = AE_EINVAL;
    }
    // (kr, vr): the sorted pairs; (kf, vf): the free pair
    uint64_t *kr = k0, *kf = k1;
    uint32_t *vr = v0, *vf = v1;
    int bits = b * L;
    int64_t h = L;
    while (res == AE_OK) {
        if (ae_radix_sort(kr, vr, kf, vf, N, bits, tmp, st)) {
            std::swap(kr, kf);
            std::swap(vr, vf);
        }
        if (rounds) ++*rounds;
        g_launches += 2;
        k_sa_heads<<<grid_for(N, 256), 256, 0, st>>>(kr, N, vf);
        const uint32_t *in[1] = {vf};
        uint64_t *out[1] = {kf};
        ae_scan_u32(in, out, 1, N, total, tmp, st);
        k_sa_rank<<<grid_for(N, 256), 256, 0, st>>>(vr, vf, kf, N, rank, bad);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(&G, total, sizeof(uint64_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            res = AE_ECUDA;
            break;
        }
        if (h_bad || G < 1 || (int64_t)G > N) {
            res = AE_ECUDA;   // not a permutation: an internal error
            break;
        }
        if ((int64_t)G == N) break;
        if (h >= N) {         // every rank is distinct once h reaches N
            res = AE_ECUDA;
            break;
        }
        const int rb = sa_bits_for(G);
        bits = rb + sa_bits_for(G - 1);
        ++g_launches;
        k_sa_pair_keys<<<grid_for(N, 256), 256, 0, st>>>(rank, N, h, rb, kf, vf);
        std::swap(kr, kf);
        std::swap(vr, vf);
        h *= 2;
    }
    if (res == AE_OK &&
        (cudaMemcpyAsync(d_sa, vr, sizeof(int32_t) * N, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
         cudaStreamSynchronize(st) != cudaSuccess))
        res = AE_ECUDA;
    if (res != AE_OK) cudaStreamSynchronize(st);
    for (void *p : {(void *)s, (void *)k0, (void *)k1, (void *)v0, (void *)v1, (void *)rank, (void *)tmp,
                    (void *)total, (void *)bad})
        if (p) cudaFree(p);
    return res;
}
