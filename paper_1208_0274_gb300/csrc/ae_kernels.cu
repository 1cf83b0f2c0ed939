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

#include "ae_kernels.h"

#define FULL 0xffffffffu

// Kernel launches issued by the calling thread (reported as ae_stats.launches).
thread_local int64_t g_launches = 0;

namespace {

// ------------------------------------------------------------------ helpers

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

__device__ __forceinline__ int64_t floordiv(int64_t a, int64_t b) {  // b > 0
    int64_t q = a / b;
    if ((a % b != 0) && (a < 0)) --q;
    return q;
}

// Theorem 2 threshold of query column j (0-based): an entry lives iff > thr.
__device__ __forceinline__ int32_t thr_of(int32_t j, int32_t m, int32_t H, int32_t g) {
    int64_t t = (int64_t)H - 1 - (int64_t)(m - 1 - j) * g;
    return t > 0 ? (int32_t)t : 0;
}

__device__ __forceinline__ int32_t delta_of(const ScoreView &sc, const int8_t *smat, int c, int q) {
    return sc.use_matrix ? (int32_t)smat[c * AE_MAX_SIGMA + q] : (c == q ? sc.sa : sc.sb);
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
    return acc;
}

template <int SIGMA>
__device__ __forceinline__ uint32_t occ_of(const IndexView &ix, int c, uint32_t k) {
    return SIGMA == 4 ? occ_dna(ix, c, k) : occ_prot(ix, c, k);
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
    o.run_len = 0;
    o.run_hits = 0;
    if (valid && incl > AE_KNEG / 2 && o.run_start < next_col) {
        const int64_t K = incl;
        int64_t x1 = floordiv(sc.sg + K - 1, u);
        int64_t x2 = floordiv(sc.sg + K - H + (int64_t)(m - 1) * g, u + g);
        int64_t xm = min(min(x1, x2), (int64_t)next_col - 1);
        int64_t r = xm - o.run_start + 1;
        if (r > 0) {
            o.run_len = (int32_t)r;
            int64_t xh = floordiv(sc.sg + K - H, u);
            int64_t rh = min(xh, (int64_t)o.run_start + r - 1) - o.run_start + 1;
            o.run_hits = rh > 0 ? (int32_t)rh : 0;
        }
    }
}

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
        aM[t] = a.d0 * a.sc.sa;
        aGa[t] = AE_NEG;
        if (flags[t]) {
            uint64_t key = keys[t];
            uint64_t gram = key & gmask;
            uint32_t lo = 0, hi = (uint32_t)(a.ix.n + 1);
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
            nd.item = (int32_t)(key >> (bits * a.d0));
            nd.cnt = 0;
            nd.off = (uint64_t)t;
            nodes[k] = nd;
        }
    }
}

__global__ void k_seed_fix(Node *nodes, const uint64_t *nn_dev, int64_t N) {
    const int64_t nn = (int64_t)*nn_dev;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nn; i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t end = (i + 1 < nn) ? nodes[i + 1].off : (uint64_t)N;
        nodes[i].cnt = (uint32_t)(end - nodes[i].off);
    }
}

// ------------------------------------------------------------------ trie expansion

// One warp per frontier node; for each letter c the child's SA range and its
// row.  The count pass sizes every child's output; the write pass recomputes
// the same row and stores it at the scanned offsets (deterministic layout).
template <int SIGMA, bool WRITE>
__global__ void __launch_bounds__(256) k_expand(ExpandArgs a) {
    __shared__ int8_t smat[AE_MAX_SIGMA * AE_MAX_SIGMA];
    load_matrix(a.sc, smat);
    const int lane = threadIdx.x & 31;
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const ScoreView &sc = a.sc;
    const int32_t u = -sc.ss, oe = sc.sg + sc.ss;
    unsigned long long st_nodes = 0, st_ent = 0, st_t[3] = {0, 0, 0};

    for (int64_t node = gw; node < a.nnodes; node += nw) {
        const Node nd = a.nodes[node];
        const WorkItem it = a.items[nd.item];
        const int qid = it.qid;
        const int32_t m = a.qv.m[qid], H = a.qv.H[qid];
        const uint8_t *P = a.qv.codes + a.qv.off[qid];
        uint32_t clo = 0, chi = 0;
        if (lane < SIGMA) {
            clo = a.ix.C[lane] + occ_of<SIGMA>(a.ix, lane, nd.lo);
            chi = a.ix.C[lane] + occ_of<SIGMA>(a.ix, lane, nd.hi);
        }
        const bool root = nd.cnt == AE_ROOT_ROW;
        const int64_t len = root ? (int64_t)(it.c1 - it.c0) : (int64_t)nd.cnt;
        if (WRITE) ++st_nodes;
        for (int c = 0; c < SIGMA; ++c) {
            const uint32_t lo_c = __shfl_sync(FULL, clo, c), hi_c = __shfl_sync(FULL, chi, c);
            const int64_t slot = node * SIGMA + c;
            if (hi_c <= lo_c || len == 0) {
                if (!WRITE && lane == 0) {
                    a.c_fr_ent[slot] = 0;
                    a.c_lf_ent[slot] = 0;
                    a.c_fr_node[slot] = 0;
                    a.c_lf_node[slot] = 0;
                    a.c_hits[slot] = 0;
                }
                continue;
            }
            const int kind = (hi_c - lo_c >= 2) ? 1 : 2;
            int32_t *oj = nullptr, *oM = nullptr, *oGa = nullptr;
            RangeHit *orh = nullptr;
            if (WRITE) {
                if (kind == 1) {
                    uint64_t o = a.o_fr_ent[slot];
                    oj = a.fj + o; oM = a.fM + o; oGa = a.fGa + o;
                    orh = a.rhits + a.hit_base + a.o_hits[slot];
                } else {
                    uint64_t o = a.lf_ent_base + a.o_lf_ent[slot];
                    oj = a.lj + o; oM = a.lM + o; oGa = a.lGa + o;
                }
            }
            uint32_t ent_run = 0, hit_run = 0;
            int32_t carry = AE_KNEG, prev_j = -2, prev_M = AE_NEG;
            for (int64_t base = 0; base < len; base += 32) {
                const int64_t idx = base + lane;
                const bool valid = idx < len;
                int32_t colA = m, MpA = AE_NEG, GaA = AE_NEG, MpB = AE_NEG, next_col = m;
                bool hasB = false;
                int tierA = 0, tierB = 0;
                int32_t Dprev = AE_NEG, Gap = AE_NEG, Dk = AE_NEG;
                if (root) {
                    if (valid) {
                        colA = it.c0 + (int32_t)idx;
                        int32_t D = delta_of(sc, smat, c, P[colA]);
                        int32_t t = thr_of(colA, m, H, sc.gmax);
                        Dprev = D > t ? D : AE_NEG;
                        MpA = Dprev;
                        next_col = (colA + 1 < it.c1) ? colA + 1 : m;
                    }
                } else {
                    int32_t j = m, M = AE_NEG, Ga = AE_NEG;
                    if (valid) {
                        j = a.pj[nd.off + idx];
                        M = a.pM[nd.off + idx];
                        Ga = a.pGa[nd.off + idx];
                    }
                    int32_t jn = __shfl_down_sync(FULL, j, 1);
                    if (lane == 31 && idx + 1 < len) jn = a.pj[nd.off + idx + 1];
                    if (idx + 1 >= len) jn = m;
                    int32_t pjv = __shfl_up_sync(FULL, j, 1), pMv = __shfl_up_sync(FULL, M, 1);
                    if (lane == 0) {
                        pjv = prev_j;
                        pMv = prev_M;
                    }
                    if (valid) {
                        colA = j;
                        const int32_t tA = thr_of(j, m, H, sc.gmax);
                        if (pjv + 1 == j && pMv > AE_NEG) {
                            int32_t D = pMv + delta_of(sc, smat, c, P[j]);
                            Dprev = D > tA ? D : AE_NEG;
                        }
                        int32_t g1 = Ga > AE_NEG ? Ga + sc.ss : AE_NEG;
                        int32_t g2 = M + oe;
                        int32_t gap = max(g1, g2);
                        Gap = gap > tA ? gap : AE_NEG;
                        MpA = max(Dprev, Gap);
                        GaA = Gap;
                        hasB = (j + 1 < m) && (j + 1 != jn);
                        if (hasB) {
                            int32_t D = M + delta_of(sc, smat, c, P[j + 1]);
                            Dk = D > thr_of(j + 1, m, H, sc.gmax) ? D : AE_NEG;
                            MpB = Dk;
                        }
                        next_col = jn;
                    }
                    prev_j = __shfl_sync(FULL, j, 31);
                    prev_M = __shfl_sync(FULL, M, 31);
                }
                // horizontal gaps: max-plus scan of keys over the slots
                int32_t keyA = MpA > AE_NEG ? MpA + colA * u : AE_KNEG;
                int32_t keyB = MpB > AE_NEG ? MpB + (colA + 1) * u : AE_KNEG;
                int32_t incl = warp_incl_max(max(keyA, keyB));
                int32_t excl = __shfl_up_sync(FULL, incl, 1);
                if (lane == 0) excl = AE_KNEG;
                incl = max(incl, carry);
                excl = max(excl, carry);
                SlotOut o;
                slot_finish(colA, MpA, hasB, MpB, next_col, excl, incl, sc, m, H, u, valid, o);
                carry = __shfl_sync(FULL, incl, 31);

                const uint32_t nA = o.aliveA, nB = o.aliveB, nR = (uint32_t)o.run_len;
                const uint32_t cnt = nA + nB + nR;
                const uint32_t hA = o.aliveA && o.MA >= H, hB = o.aliveB && o.MB >= H;
                const uint32_t hcnt = kind == 1 ? (hA + hB + (uint32_t)o.run_hits) : 0u;
                const uint32_t ci = warp_incl_sum(cnt), hi = warp_incl_sum(hcnt);
                const uint32_t ctot = __shfl_sync(FULL, ci, 31), htot = __shfl_sync(FULL, hi, 31);
                if (WRITE) {
                    const uint32_t e0 = ent_run + ci - cnt, h0 = hit_run + hi - hcnt;
                    if (o.aliveA) {
                        oj[e0] = colA;
                        oM[e0] = o.MA;
                        oGa[e0] = GaA;
                        tierA = (Dprev > AE_NEG) + (Gap > AE_NEG) + (o.GbA > thr_of(colA, m, H, sc.gmax));
                        st_t[max(tierA, 1) - 1]++;
                    }
                    if (o.aliveB) {
                        oj[e0 + nA] = colA + 1;
                        oM[e0 + nA] = o.MB;
                        oGa[e0 + nA] = AE_NEG;
                        tierB = (Dk > AE_NEG) + (o.GbB > thr_of(colA + 1, m, H, sc.gmax));
                        st_t[max(tierB, 1) - 1]++;
                    }
                    st_t[0] += nR;
                    if (kind == 1) {
                        uint32_t hp = h0;
                        if (hA) {
                            RangeHit r = {lo_c, hi_c, qid, colA, o.MA, 0};
                            orh[hp++] = r;
                        }
                        if (hB) {
                            RangeHit r = {lo_c, hi_c, qid, colA + 1, o.MB, 0};
                            orh[hp++] = r;
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
                        const uint32_t d0 = __shfl_sync(FULL, e0 + nA + nB, L);
                        const uint32_t hd = __shfl_sync(FULL, h0 + hA + hB, L);
                        for (int32_t t = lane; t < rl; t += 32) {
                            const int32_t col = s0 + t;
                            const int32_t v = sc.sg - col * u + K;
                            oj[d0 + t] = col;
                            oM[d0 + t] = v;
                            oGa[d0 + t] = AE_NEG;
                            if (kind == 1 && t < rh) {
                                RangeHit r = {lo_c, hi_c, qid, col, v, 0};
                                orh[hd + t] = r;
                            }
                        }
                    }
                }
                ent_run += ctot;
                hit_run += htot;
            }
            if (WRITE) {
                st_ent += ent_run;
                if (lane == 0 && ent_run > 0) {
                    if (kind == 1) {
                        Node cn;
                        cn.lo = lo_c;
                        cn.hi = hi_c;
                        cn.item = nd.item;
                        cn.cnt = ent_run;
                        cn.off = a.o_fr_ent[slot];
                        a.fnodes[a.o_fr_node[slot]] = cn;
                    } else {
                        Inject in;
                        in.qid = qid;
                        in.e = a.ix.tend[lo_c];
                        in.cnt = ent_run;
                        in.pad = 0;
                        in.off = a.lf_ent_base + a.o_lf_ent[slot];
                        a.inj[a.lf_node_base + a.o_lf_node[slot]] = in;
                    }
                }
            } else if (lane == 0) {
                a.c_fr_ent[slot] = kind == 1 ? ent_run : 0u;
                a.c_lf_ent[slot] = kind == 2 ? ent_run : 0u;
                a.c_fr_node[slot] = (kind == 1 && ent_run > 0) ? 1u : 0u;
                a.c_lf_node[slot] = (kind == 2 && ent_run > 0) ? 1u : 0u;
                a.c_hits[slot] = hit_run;
            }
        }
    }
    if (WRITE && a.stats) {
        // per-lane tier counts, lane 0 holds node/entry counts (warp-uniform)
        unsigned long long t0 = st_t[0], t1 = st_t[1], t2 = st_t[2];
        for (int d = 16; d > 0; d >>= 1) {
            t0 += __shfl_down_sync(FULL, t0, d);
            t1 += __shfl_down_sync(FULL, t1, d);
            t2 += __shfl_down_sync(FULL, t2, d);
        }
        if (lane == 0) {
            if (st_nodes) atomicAdd(&a.stats->nodes, st_nodes);
            if (st_ent) atomicAdd(&a.stats->entries, st_ent);
            if (t0) atomicAdd(&a.stats->tier[0], t0);
            if (t1) atomicAdd(&a.stats->tier[1], t1);
            if (t2) atomicAdd(&a.stats->tier[2], t2);
        }
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

// One warp per segment of `seg` consecutive injections (sorted by query and
// text end).  The warp carries a row R along text positions p, p+1, ...:
//   candidates of row p+1 = the vertical and diagonal slots generated from R
//   with letter T[p+1], merged by maximum with every injected row at p+1;
//   then the horizontal-gap finish of Section 2.2 gives row p+1.
// The walk jumps to the next injection when R has no live entry.  Rows live
// in per-warp global scratch (cap entries per buffer); a row that outgrows it
// sets leaf_overflow and the host reruns with a larger cap.
__global__ void __launch_bounds__(128) k_leaf(LeafArgs a) {
    __shared__ int8_t smat[AE_MAX_SIGMA * AE_MAX_SIGMA];
    load_matrix(a.sc, smat);
    const int lane = threadIdx.x & 31;
    const int gw = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    if (gw >= a.nwarps) return;
    const ScoreView &sc = a.sc;
    const int32_t u = -sc.ss, oe = sc.sg + sc.ss, g = sc.gmax;
    const int64_t cap = a.cap;
    int32_t *wb = a.scratch + (int64_t)gw * 12 * cap;
    Buf R = {wb, wb + cap, wb + 2 * cap};
    Buf Rn = {wb + 3 * cap, wb + 4 * cap, wb + 5 * cap};
    Buf Cb = {wb + 6 * cap, wb + 7 * cap, wb + 8 * cap};
    Buf C2 = {wb + 9 * cap, wb + 10 * cap, wb + 11 * cap};
    const uint64_t jmask = (1ull << a.bj) - 1ull;
    unsigned long long st_rows = 0, st_ent = 0, st_t[3] = {0, 0, 0};
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
        while (true) {
            int64_t clen = 0;
            if (rlen == 0) {
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
                ++p;
                if (p >= a.ix.n) break;
                const int c = a.ix.text[p];
                // ---- generate slots from R with letter c
                int32_t prev_j = -2, prev_M = AE_NEG;
                for (int64_t base = 0; base < rlen; base += 32) {
                    const int64_t idx = base + lane;
                    const bool valid = idx < rlen;
                    int32_t j = m, M = AE_NEG, Ga = AE_NEG;
                    if (valid) {
                        j = R.j[idx];
                        M = R.M[idx];
                        Ga = R.Ga[idx];
                    }
                    int32_t jn = __shfl_down_sync(FULL, j, 1);
                    if (lane == 31 && idx + 1 < rlen) jn = R.j[idx + 1];
                    if (idx + 1 >= rlen) jn = m;
                    int32_t pjv = __shfl_up_sync(FULL, j, 1), pMv = __shfl_up_sync(FULL, M, 1);
                    if (lane == 0) {
                        pjv = prev_j;
                        pMv = prev_M;
                    }
                    int32_t MpA = AE_NEG, GaA = AE_NEG, MpB = AE_NEG;
                    if (valid) {
                        const int32_t tA = thr_of(j, m, H, g);
                        int32_t Dp = AE_NEG;
                        if (pjv + 1 == j && pMv > AE_NEG) Dp = pMv + delta_of(sc, smat, c, P[j]);
                        int32_t gap = max(Ga > AE_NEG ? Ga + sc.ss : AE_NEG, M + oe);
                        GaA = gap > tA ? gap : AE_NEG;
                        Dp = Dp > tA ? Dp : AE_NEG;
                        MpA = max(Dp, GaA);
                        if (j + 1 < m && j + 1 != jn) {
                            int32_t D = M + delta_of(sc, smat, c, P[j + 1]);
                            MpB = D > thr_of(j + 1, m, H, g) ? D : AE_NEG;
                        }
                    }
                    const uint32_t oA = MpA > AE_NEG, oB = MpB > AE_NEG;
                    const uint32_t cn = oA + oB;
                    const uint32_t ci = warp_incl_sum(cn);
                    const uint32_t tot = __shfl_sync(FULL, ci, 31);
                    if (clen + tot > cap) {
                        overflow = true;
                        break;
                    }
                    const int64_t d = clen + ci - cn;
                    if (oA) {
                        Cb.j[d] = j;
                        Cb.M[d] = MpA;
                        Cb.Ga[d] = GaA;
                    }
                    if (oB) {
                        Cb.j[d + oA] = j + 1;
                        Cb.M[d + oA] = MpB;
                        Cb.Ga[d + oA] = AE_NEG;
                    }
                    clen += tot;
                    prev_j = __shfl_sync(FULL, j, 31);
                    prev_M = __shfl_sync(FULL, M, 31);
                }
                __syncwarp();
                if (overflow) break;
            }
            // ---- merge the rows injected at (qid, p)
            while (k < kend) {
                const Inject I = a.inj[a.order[k]];
                if (I.qid != qid || I.e != p) break;
                ++k;
                const int32_t *ij = a.lj + I.off, *iM = a.lM + I.off, *iGa = a.lGa + I.off;
                const int64_t icnt = I.cnt;
                if (clen + icnt > cap) {
                    overflow = true;
                    break;
                }
                for (int64_t base = 0; base < clen; base += 32) {
                    const int64_t idx = base + lane;
                    if (idx < clen) {
                        const int32_t x = Cb.j[idx];
                        const int64_t d = idx + lower_bound_g(ij, icnt, x);
                        C2.j[d] = x;
                        C2.M[d] = Cb.M[idx];
                        C2.Ga[d] = Cb.Ga[idx];
                    }
                }
                for (int64_t base = 0; base < icnt; base += 32) {
                    const int64_t idx = base + lane;
                    if (idx < icnt) {
                        const int32_t y = ij[idx];
                        const int64_t d = idx + upper_bound_g(Cb.j, clen, y);
                        C2.j[d] = y;
                        C2.M[d] = iM[idx];
                        C2.Ga[d] = iGa[idx];
                    }
                }
                __syncwarp();
                const int64_t len2 = clen + icnt;
                int64_t out = 0;
                for (int64_t base = 0; base < len2; base += 32) {
                    const int64_t idx = base + lane;
                    const bool valid = idx < len2;
                    int32_t j = 0, Mv = AE_NEG, Gv = AE_NEG;
                    bool keep = false;
                    if (valid) {
                        j = C2.j[idx];
                        Mv = C2.M[idx];
                        Gv = C2.Ga[idx];
                        keep = !(idx > 0 && C2.j[idx - 1] == j);
                        if (idx + 1 < len2 && C2.j[idx + 1] == j) {
                            Mv = max(Mv, C2.M[idx + 1]);
                            Gv = max(Gv, C2.Ga[idx + 1]);
                        }
                    }
                    const uint32_t ci = warp_incl_sum(keep ? 1u : 0u);
                    const uint32_t tot = __shfl_sync(FULL, ci, 31);
                    __syncwarp();
                    if (keep) {
                        const int64_t d = out + ci - 1;
                        Cb.j[d] = j;
                        Cb.M[d] = Mv;
                        Cb.Ga[d] = Gv;
                    }
                    out += tot;
                }
                clen = out;
                __syncwarp();
            }
            if (overflow) break;
            // ---- finish: horizontal gaps, prune, hits -> Rn
            int64_t nlen = 0;
            int32_t carry = AE_KNEG;
            for (int64_t base = 0; base < clen; base += 32) {
                const int64_t idx = base + lane;
                const bool valid = idx < clen;
                int32_t col = m, Mp = AE_NEG, Ga = AE_NEG;
                if (valid) {
                    col = Cb.j[idx];
                    Mp = Cb.M[idx];
                    Ga = Cb.Ga[idx];
                }
                int32_t nc = __shfl_down_sync(FULL, col, 1);
                if (lane == 31 && idx + 1 < clen) nc = Cb.j[idx + 1];
                if (idx + 1 >= clen) nc = m;
                const int32_t key = Mp > AE_NEG ? Mp + col * u : AE_KNEG;
                int32_t incl = warp_incl_max(key);
                int32_t excl = __shfl_up_sync(FULL, incl, 1);
                if (lane == 0) excl = AE_KNEG;
                incl = max(incl, carry);
                excl = max(excl, carry);
                SlotOut o;
                slot_finish(col, Mp, false, AE_NEG, nc, excl, incl, sc, m, H, u, valid, o);
                carry = __shfl_sync(FULL, incl, 31);
                const uint32_t nA = o.aliveA, nR = (uint32_t)o.run_len;
                const uint32_t cn = nA + nR;
                const uint32_t ci = warp_incl_sum(cn);
                const uint32_t tot = __shfl_sync(FULL, ci, 31);
                if (nlen + tot > cap) {
                    overflow = true;
                    break;
                }
                const uint32_t hA = o.aliveA && o.MA >= H;
                const uint32_t hc = hA + (uint32_t)o.run_hits;
                const uint32_t hi = warp_incl_sum(hc);
                const uint32_t htot = __shfl_sync(FULL, hi, 31);
                unsigned long long hbase = 0;
                if (htot) {
                    if (lane == 0) hbase = atomicAdd(a.hit_count, (unsigned long long)htot);
                    hbase = __shfl_sync(FULL, hbase, 0);
                }
                const bool hok = hbase + htot <= a.hit_cap;
                const uint64_t kq = ((uint64_t)qid << (a.be + a.bj)) | ((uint64_t)(uint32_t)p << a.bj);
                const int64_t e0 = nlen + ci - cn;
                const uint64_t h0 = hbase + hi - hc;
                if (o.aliveA) {
                    Rn.j[e0] = col;
                    Rn.M[e0] = o.MA;
                    Rn.Ga[e0] = Ga;
                    int tier = (Mp > AE_NEG) + (Ga > AE_NEG) + (o.GbA > thr_of(col, m, H, g));
                    st_t[min(max(tier, 1), 3) - 1]++;
                    if (hA && hok) {
                        a.hit_key[h0] = kq | ((uint64_t)col & jmask);
                        a.hit_score[h0] = o.MA;
                    }
                }
                st_t[0] += nR;
                unsigned rmask = __ballot_sync(FULL, nR > 0);
                while (rmask) {
                    const int L = __ffs(rmask) - 1;
                    rmask &= rmask - 1;
                    const int32_t s0 = __shfl_sync(FULL, o.run_start, L);
                    const int32_t rl = __shfl_sync(FULL, o.run_len, L);
                    const int32_t rh = __shfl_sync(FULL, o.run_hits, L);
                    const int32_t K = __shfl_sync(FULL, incl, L);
                    const int64_t d0 = __shfl_sync(FULL, e0 + nA, L);
                    const uint64_t hd = __shfl_sync(FULL, h0 + hA, L);
                    for (int32_t t = lane; t < rl; t += 32) {
                        const int32_t cc = s0 + t;
                        const int32_t v = sc.sg - cc * u + K;
                        Rn.j[d0 + t] = cc;
                        Rn.M[d0 + t] = v;
                        Rn.Ga[d0 + t] = AE_NEG;
                        if (t < rh && hok) {
                            a.hit_key[hd + t] = kq | ((uint64_t)cc & jmask);
                            a.hit_score[hd + t] = v;
                        }
                    }
                }
                if (!hok && lane == 0) atomicAdd(&a.stats->hit_overflow, 1ull);
                nlen += tot;
            }
            __syncwarp();
            if (overflow) break;
            Buf t = R;
            R = Rn;
            Rn = t;
            rlen = nlen;
            ++st_rows;
            st_ent += (unsigned long long)nlen;
        }
        if (overflow && lane == 0) atomicAdd(&a.stats->leaf_overflow, 1ull);
    }
    unsigned long long t0 = st_t[0], t1 = st_t[1], t2 = st_t[2];
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

__global__ void k_unique_flags(const uint64_t *key, int64_t N, uint32_t *flags) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N; t += (int64_t)gridDim.x * blockDim.x)
        flags[t] = (t == 0 || key[t] != key[t - 1]) ? 1u : 0u;
}

__global__ void k_unique_write(const uint64_t *key, const int32_t *score, int64_t N, const uint64_t *off, int be,
                               int bj, ae_hit *out, unsigned long long *qcount) {
    const uint64_t jmask = (1ull << bj) - 1ull, emask = (1ull << be) - 1ull;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N; t += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = key[t];
        if (t > 0 && key[t - 1] == k) continue;
        int32_t best = score[t];
        for (int64_t u = t + 1; u < N && key[u] == k; ++u) best = max(best, score[u]);
        ae_hit h;
        h.text_end = (int64_t)((k >> bj) & emask);
        h.query_end = (int32_t)(k & jmask);
        h.score = best;
        out[off[t]] = h;
        atomicAdd(&qcount[k >> (be + bj)], 1ull);
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

void ae_expand(const ExpandArgs &a, bool write, cudaStream_t st) {
    if (a.nnodes <= 0) return;
    const int threads = 256;
    const unsigned blocks = grid_for(a.nnodes * 32, threads, 152 * 16);
    if (a.ix.sigma == 4) {
        if (write) { ++g_launches; k_expand<4, true><<<blocks, threads, 0, st>>>(a); }
        else { ++g_launches; k_expand<4, false><<<blocks, threads, 0, st>>>(a); }
    } else {
        if (write) { ++g_launches; k_expand<20, true><<<blocks, threads, 0, st>>>(a); }
        else { ++g_launches; k_expand<20, false><<<blocks, threads, 0, st>>>(a); }
    }
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

void ae_unique_flags(const uint64_t *key, int64_t N, uint32_t *flags, cudaStream_t st) {
    if (N <= 0) return;
    ++g_launches;
    k_unique_flags<<<grid_for(N, 256), 256, 0, st>>>(key, N, flags);
}

void ae_unique_write(const uint64_t *key, const int32_t *score, int64_t N, const uint64_t *flag_off, int be, int bj,
                     ae_hit *out, unsigned long long *qcount, cudaStream_t st) {
    if (N <= 0) return;
    ++g_launches;
    k_unique_write<<<grid_for(N, 256), 256, 0, st>>>(key, score, N, flag_off, be, bj, out, qcount);
}
