// Host orchestration of the search and the C ABI of include/ae.h.
//
// ae_search_device runs, per batch of work items:
//   seed (Theorem 3: the query's (q-1)-grams located by backward search) or
//   the trie root;  then one trie level per iteration (DNA: one launch that
//   counts, reserves and writes; general route: count pass, scan, write pass)
//   until the frontier is empty;  then the text-position sweep over the
//   rows that reached a single occurrence;  then the located hits of the
//   multi-occurrence nodes.  All hits of all batches are sorted by
//   (query, text end, query end) and reduced to the per-cell maximum
//   (Algorithm 1's per-cell maximum and hit report).
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <atomic>
#include <mutex>
#include <new>
#include <system_error>
#include <thread>
#include <vector>

#include "ae_internal.h"
#include "ae_kernels.h"

namespace {

thread_local ae_stats g_last_stats;

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    bool carved = false;   // points into the static scratch of ae_search_device_static
};

// Set only inside ae_search_device_static: buffers are then carved from the
// static device array instead of allocated (see the end of this file).
struct StaticArena {
    char *base;
    size_t cap;
    size_t used;
};
thread_local StaticArena *g_arena = nullptr;
// Largest sweep row (entries) the no-allocation entry point retries with.
constexpr int32_t AE_STATIC_MAX_LEAF_CAP = 1024;

void carve(DevBuf &b, size_t bytes, size_t keep, cudaStream_t st);

struct ae_error {
    ae_status st;
};

#define CU(x)                                    \
    do {                                         \
        cudaError_t _e = (x);                    \
        if (_e != cudaSuccess) throw ae_error{AE_ECUDA}; \
    } while (0)

std::atomic<int64_t> g_ws_bytes{0};   // device bytes held by all workspaces of the process
bool mem_trace() {
    static int on = -1;
    if (on < 0) on = getenv("AE_TRACE_MEM") != nullptr;
    return on == 1;
}
bool trace() {
    static int on = -1;
    if (on < 0) on = getenv("AE_TRACE") != nullptr;
    return on == 1;
}
void trace_alloc(size_t nb, bool ok) {
    if (!mem_trace()) return;
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    fprintf(stderr, "[ae mem] alloc %.3f GB %s; workspaces hold %.3f GB; device free %.3f of %.3f GB\n", nb / 1e9,
            ok ? "ok" : "FAILED", g_ws_bytes.load() / 1e9, fr / 1e9, tot / 1e9);
}

// Optional cap on the device bytes of the running search's workspace
// (ae_options.workspace_limit): growth past it fails as AE_ENOMEM.
thread_local int64_t g_ws_limit = 0;
int64_t cur_ws_bytes();

void check_limit(const DevBuf &b, size_t nb) {
    if (g_ws_limit > 0 && cur_ws_bytes() - (int64_t)b.bytes + (int64_t)nb > g_ws_limit) throw ae_error{AE_ENOMEM};
}

// Grow-only device buffer; contents are not preserved.
void ensure(DevBuf &b, size_t bytes, cudaStream_t st) {
    if (bytes <= b.bytes) return;
    if (g_arena) {
        carve(b, bytes, 0, st);
        return;
    }
    size_t nb = std::max(bytes, b.bytes + b.bytes / 4);
    nb = (nb + 255) & ~size_t(255);
    check_limit(b, nb);
    if (b.p) {
        CU(cudaStreamSynchronize(st));
        CU(cudaFree(b.p));
        g_ws_bytes -= (int64_t)b.bytes;
        b.p = nullptr;
        b.bytes = 0;
    }
    if (cudaMalloc(&b.p, nb) != cudaSuccess) {
        cudaGetLastError();
        trace_alloc(nb, false);
        throw ae_error{AE_ENOMEM};
    }
    g_ws_bytes += (int64_t)nb;
    trace_alloc(nb, true);
    b.bytes = nb;
}

// Grow preserving the first `keep` bytes.
void ensure_keep(DevBuf &b, size_t bytes, size_t keep, cudaStream_t st) {
    if (bytes <= b.bytes) return;
    if (g_arena) {
        carve(b, bytes, keep, st);
        return;
    }
    size_t nb = std::max(bytes, b.bytes + b.bytes / 4);
    nb = (nb + 255) & ~size_t(255);
    check_limit(b, nb);
    void *p = nullptr;
    if (cudaMalloc(&p, nb) != cudaSuccess) {
        cudaGetLastError();
        trace_alloc(nb, false);
        throw ae_error{AE_ENOMEM};
    }
    g_ws_bytes += (int64_t)nb;
    trace_alloc(nb, true);
    if (b.p) {
        if (keep) CU(cudaMemcpyAsync(p, b.p, keep, cudaMemcpyDeviceToDevice, st));
        CU(cudaStreamSynchronize(st));
        CU(cudaFree(b.p));
        g_ws_bytes -= (int64_t)b.bytes;
    }
    b.p = p;
    b.bytes = nb;
}

template <typename T>
T *ptr(DevBuf &b) {
    return reinterpret_cast<T *>(b.p);
}

// Upload a level's starting counters, leaving the device's overflow flag as it
// is: a disagreement reported by any earlier pass of the batch stays visible.
void upload_level_counters(LevelCounters *d, const LevelCounters &h, cudaStream_t st) {
    const size_t ov = offsetof(LevelCounters, overflow);
    CU(cudaMemcpyAsync(d, &h, ov, cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync((char *)d + ov + 8, (const char *)&h + ov + 8, sizeof(LevelCounters) - ov - 8,
                       cudaMemcpyHostToDevice, st));
}


struct Workspace {
    cudaStream_t stream = nullptr;
    // queries
    DevBuf ascii, codes, qoff, qm, qH, items, item_pos, bad;
    // level arenas (ping-pong) and nodes
    DevBuf aj[2], aM[2], aGa[2], nodes[2];
    // count outputs and scanned offsets (5 arrays each)
    DevBuf cnt[5], off[5], totals, scan_tmp;
    // leaf arena, injections, range hits
    DevBuf lj, lM, lGa, inj, rhits;
    // sort buffers
    DevBuf sk0, sv0, sk1, sv1, sort_tmp;
    // point hits of the whole search
    DevBuf hkey, hscore, hcount, hk1, hv1;
    // leaf sweep scratch; walks handed on to blocks (state, count, row buffers)
    DevBuf scratch, next_seg, esc, esc_count, esc_rows;
    // walk layout of the DNA row kernel: per warp and lane, the count phase's child rows
    DevBuf stage;
    // output
    DevBuf uniq, uflags, uoff, qcount;
    DevBuf stats, segs, ctr, seg_cnt, seg_hit, task_first, task_tot, task_off, task_tmp, task_sum, res, res_key;
    double fr_ratio = 1.2, lf_ratio = 0.6, hit_ratio = 0.5;
    // pinned host staging
    uint64_t *h_tot = nullptr;
    bool h_tot_static = false;
    uint8_t *h_stage = nullptr;   // pinned copy of the ASCII queries of ae_search (grow-only)
    size_t h_stage_bytes = 0;
    // the threaded result copy of ae_search: two pinned chunks, one stream and two
    // events per copying thread, and the event that orders them after the search
    uint8_t *h_out = nullptr;
    size_t h_out_bytes = 0;
    std::vector<cudaStream_t> out_st;
    std::vector<cudaEvent_t> out_ev;
    cudaEvent_t out_ready = nullptr;
    int32_t leaf_cap = 0;
    std::mutex busy;              // one search at a time per workspace (per stream)

    int64_t device_bytes() {
        int64_t t = 0;
        for (DevBuf *b : bufs())
            if (!b->carved) t += (int64_t)b->bytes;
        return t;
    }

    std::vector<DevBuf *> bufs() {
        return {&ascii, &codes, &qoff, &qm, &qH, &items, &item_pos, &bad, &aj[0], &aj[1], &aM[0],
                &aM[1], &aGa[0], &aGa[1], &nodes[0], &nodes[1], &cnt[0], &cnt[1], &cnt[2], &cnt[3],
                &cnt[4], &off[0], &off[1], &off[2], &off[3], &off[4], &totals, &scan_tmp, &lj, &lM,
                &lGa, &inj, &rhits, &sk0, &sv0, &sk1, &sv1, &sort_tmp, &hkey, &hscore, &hcount, &hk1,
                &hv1, &scratch, &next_seg, &esc, &esc_count, &esc_rows, &stage, &uniq, &uflags, &uoff, &qcount, &stats, &segs, &ctr, &seg_cnt, &seg_hit,
                &task_first, &task_tot, &task_off, &task_tmp, &task_sum, &res, &res_key};
    }

    ~Workspace() {
        for (DevBuf *b : bufs())
            if (b->p && !b->carved) {
                cudaFree(b->p);
                g_ws_bytes -= (int64_t)b->bytes;
            }
        if (h_tot && !h_tot_static) cudaFreeHost(h_tot);
        if (h_stage) cudaFreeHost(h_stage);
        if (h_out) cudaFreeHost(h_out);
        for (cudaStream_t s : out_st) cudaStreamDestroy(s);
        for (cudaEvent_t e : out_ev) cudaEventDestroy(e);
        if (out_ready) cudaEventDestroy(out_ready);
    }

    // Free the buffers of one batch's walk (kept: queries, counters and the point
    // hits collected so far), before a batch is retried in smaller parts.
    void trim_batch() {
        DevBuf *drop[] = {&aj[0], &aj[1], &aM[0], &aM[1], &aGa[0], &aGa[1], &nodes[0], &nodes[1], &cnt[0], &cnt[1],
                          &cnt[2], &cnt[3], &cnt[4], &off[0], &off[1], &off[2], &off[3], &off[4], &scan_tmp, &lj,
                          &lM, &lGa, &inj, &rhits, &sk0, &sv0, &sk1, &sv1, &sort_tmp, &hk1, &hv1, &scratch, &esc_rows,
                          &uniq,
                          &uflags, &uoff, &segs, &seg_cnt, &seg_hit, &task_first, &task_tot, &task_off, &task_tmp,
                          &res, &res_key};
        for (DevBuf *b : drop)
            if (b->p && !b->carved) {
                cudaFree(b->p);
                g_ws_bytes -= (int64_t)b->bytes;
                b->p = nullptr;
                b->bytes = 0;
            }
        leaf_cap = 0;
    }

    // Forget every carved buffer (the next static call carves them again).
    void forget_carved() {
        for (DevBuf *b : bufs()) {
            b->p = nullptr;
            b->bytes = 0;
            b->carved = false;
        }
    }
};

thread_local Workspace *g_cur_ws = nullptr;   // workspace of the running search (limit accounting)
int64_t cur_ws_bytes() { return g_cur_ws ? g_cur_ws->device_bytes() : 0; }

}  // namespace

struct ae_index {
    HostIndex host;
    IndexView view;
    void *d_occ = nullptr, *d_tend = nullptr, *d_text = nullptr, *d_sep = nullptr, *d_ends = nullptr;
    uint32_t *d_dom[13] = {};   // q-prefix domination tables by seed depth (built on first use)
    int64_t device_bytes = 0;
    int device = 0;
    std::mutex mu;
    std::vector<std::pair<cudaStream_t, Workspace *>> ws;

    ~ae_index() {
        for (auto &p : ws) delete p.second;
        if (d_occ) cudaFree(d_occ);
        if (d_tend) cudaFree(d_tend);
        if (d_text) cudaFree(d_text);
        if (d_sep) cudaFree(d_sep);
        if (d_ends) cudaFree(d_ends);
        for (uint32_t *t : d_dom)
            if (t) cudaFree(t);
        ae_host_index_free(&host);
    }
};

const IndexView *ae_index_view(const ae_index *idx) { return &idx->view; }

namespace {

Workspace *workspace_for(const ae_index *cidx, cudaStream_t st) {
    ae_index *idx = const_cast<ae_index *>(cidx);
    std::lock_guard<std::mutex> g(idx->mu);
    for (auto &p : idx->ws)
        if (p.first == st) return p.second;
    Workspace *w = new Workspace();
    w->stream = st;
    if (cudaMallocHost(&w->h_tot, 64 * sizeof(uint64_t)) != cudaSuccess) {
        cudaGetLastError();
        delete w;
        throw ae_error{AE_ENOMEM};
    }
    idx->ws.push_back({st, w});
    return w;
}

// The q-prefix domination table of seed depth d0 (NULL when the table would be
// too large or cannot be built; the filter is then off).  Built once per index
// and depth, on `st`, and finished before any search uses it.
const uint32_t *dom_table(const ae_index *cidx, int d0, cudaStream_t st) {
    ae_index *idx = const_cast<ae_index *>(cidx);
    const int bits = idx->view.sigma == 4 ? 2 : 5;
    if (d0 < 1 || d0 > 12 || bits * d0 > 24 || idx->view.n < d0) return nullptr;
    std::lock_guard<std::mutex> g(idx->mu);
    if (idx->d_dom[d0]) return idx->d_dom[d0];
    const size_t bytes = sizeof(uint32_t) << (bits * d0);
    uint32_t *t = nullptr;
    if (cudaMalloc(&t, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (cudaMemsetAsync(t, 0, bytes, st) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(t);
        return nullptr;
    }
    ae_dom_table(idx->view, d0, t, st);
    if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
        cudaFree(t);
        return nullptr;
    }
    idx->d_dom[d0] = t;
    return t;
}

ae_status upload_index(ae_index *idx) {
    HostIndex &h = idx->host;
    size_t occ_b = sizeof(uint32_t) * (size_t)(h.nblocks * h.block_words);
    size_t tend_b = sizeof(int32_t) * (size_t)h.rows;
    size_t text_b = (size_t)h.n;
    size_t sep_b = h.nseq ? sizeof(uint32_t) * (size_t)(h.nblocks * AE_SEP_BLOCK_WORDS) : 0;
    size_t ends_b = h.nseq ? sizeof(uint32_t) * (size_t)((h.n + 31) / 32) : 0;
    if (cudaGetDevice(&idx->device) != cudaSuccess) return AE_ECUDA;
    if (cudaMalloc(&idx->d_occ, occ_b) != cudaSuccess || cudaMalloc(&idx->d_tend, tend_b) != cudaSuccess ||
        cudaMalloc(&idx->d_text, text_b) != cudaSuccess ||
        (h.nseq && (cudaMalloc(&idx->d_sep, sep_b) != cudaSuccess || cudaMalloc(&idx->d_ends, ends_b) != cudaSuccess))) {
        cudaGetLastError();
        return AE_ENOMEM;
    }
    if (cudaMemcpy(idx->d_occ, h.occ, occ_b, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(idx->d_tend, h.tend, tend_b, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(idx->d_text, h.text, text_b, cudaMemcpyHostToDevice) != cudaSuccess ||
        (h.nseq && (cudaMemcpy(idx->d_sep, h.sep, sep_b, cudaMemcpyHostToDevice) != cudaSuccess ||
                    cudaMemcpy(idx->d_ends, h.ends, ends_b, cudaMemcpyHostToDevice) != cudaSuccess)))
        return AE_ECUDA;
    idx->device_bytes = (int64_t)(occ_b + tend_b + text_b + sep_b + ends_b);
    IndexView &v = idx->view;
    memset(&v, 0, sizeof(v));
    v.occ = (const uint32_t *)idx->d_occ;
    v.tend = (const int32_t *)idx->d_tend;
    v.text = (const uint8_t *)idx->d_text;
    v.n = h.n;
    v.dollar_row = h.dollar_row;
    for (int c = 0; c <= h.sigma; ++c) v.C[c] = h.C[c];
    v.sigma = h.sigma;
    v.alphabet = h.alphabet;
    v.rows = h.rows;
    v.sep = (const uint32_t *)idx->d_sep;
    v.ends = (const uint32_t *)idx->d_ends;
    return AE_OK;
}

int bits_for(int64_t maxval) {  // bits to hold values in [0, maxval]
    int b = 1;
    while (b < 63 && (maxval >> b) != 0) ++b;
    return b;
}

double ms_since(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

ae_status make_score(const ae_scoring *s, int sigma, ScoreView &sc) {
    if (!s) return AE_EINVAL;
    memset(&sc, 0, sizeof(sc));
    sc.sg = s->gap_open;
    sc.ss = s->gap_extend;
    if (s->gap_open > 0 || s->gap_extend >= 0) return AE_EINVAL;
    if (s->matrix) {
        sc.use_matrix = 1;
        int gmax = INT32_MIN;
        for (int a = 0; a < sigma; ++a)
            for (int b = 0; b < sigma; ++b) {
                int8_t v = s->matrix[a * sigma + b];
                sc.mat[a * AE_MAX_SIGMA + b] = v;
                gmax = std::max(gmax, (int)v);
            }
        for (int a = 0; a < sigma; ++a)
            if (s->matrix[a * sigma + a] <= 0) return AE_EINVAL;
        sc.gmax = gmax;
        sc.sa = gmax;
        sc.sb = -1;
    } else {
        if (s->match <= 0 || s->mismatch >= 0) return AE_EINVAL;
        sc.sa = s->match;
        sc.sb = s->mismatch;
        sc.gmax = s->match;
        for (int a = 0; a < sigma; ++a)
            for (int b = 0; b < sigma; ++b) sc.mat[a * AE_MAX_SIGMA + b] = (int8_t)(a == b ? s->match : s->mismatch);
    }
    return AE_OK;
}

// Eq. 2 and the seed depth: the walk may start at depth q-1 (every live entry
// there is an exact match of the query's (q-1)-gram, Theorem 3), and must start
// below ceil(H/s_a) so that no hit is skipped.
int seed_depth(const ScoreView &sc, int32_t Hmin, bool qprefix) {
    if (sc.use_matrix || !qprefix) return 0;
    int q = std::min(-sc.sb, -(sc.sg + sc.ss)) / sc.sa + 1;
    int hd = (Hmin + sc.sa - 1) / sc.sa - 1;
    int d0 = std::min(q - 1, hd);
    int bits = 2;
    while (d0 > 0 && bits * d0 > 40) --d0;
    return std::max(d0, 0);
}

// Device time of kernel groups, from CUDA events recorded on the search's
// stream around each launch group (only with ae_options.profile).
struct Prof {
    bool on = false;
    cudaStream_t st = nullptr;
    std::vector<cudaEvent_t> ev[5];
    void mark(int k) {
        if (!on) return;
        cudaEvent_t e;
        CU(cudaEventCreate(&e));
        CU(cudaEventRecord(e, st));
        ev[k].push_back(e);
    }
    double ms(int k) {
        double t = 0;
        for (size_t i = 0; i + 1 < ev[k].size(); i += 2) {
            float f = 0;
            cudaEventElapsedTime(&f, ev[k][i], ev[k][i + 1]);
            t += f;
        }
        return t;
    }
    ~Prof() {
        for (auto &v : ev)
            for (cudaEvent_t e : v) cudaEventDestroy(e);
    }
};
enum { K_EXPAND = 0, K_LEAF = 1, K_SORT = 2, K_OTHER = 3, K_ROWS = 4 };

struct Search {
    const ae_index *idx;
    Workspace *w;
    cudaStream_t st;
    IndexView ix;
    ScoreView sc;
    QueryView qv;
    int32_t nq;
    std::vector<int64_t> off;
    std::vector<int32_t> m, H;
    ae_options opt;
    int be, bj, bq;
    int d0;
    int64_t nhits = 0;        // point hits accumulated in w->hkey/hscore
    double batch_hint = -1;   // expected sweep hit records of the current batch (< 0: no hints)
    ae_stats stats;
    int64_t dna_nodes = 0, dna_entries = 0, dna_retries = 0;   // DNA int16x2 route (counted on the host)
    double dna_ratio[5] = {0, 0, 0, 0, 0};   // the last DNA level's outputs per input, by arena kind
    bool dna_ratio_ok = false;
    // every batch so far held whole queries, later than the previous batch's: the
    // batches' compacted hits then already lie sorted by (query, text end, query end)
    bool batches_ordered = true;
    int32_t last_batch_q = -1;
    int num_sms = 152;
    Prof prof;

    uint64_t *tot() { return w->h_tot; }

    void sync() { CU(cudaStreamSynchronize(st)); }

    // Append `n` point hits capacity.
    void hits_reserve(int64_t extra) {
        size_t need = (size_t)(nhits + extra);
        ensure_keep(w->hkey, need * sizeof(uint64_t), (size_t)nhits * sizeof(uint64_t), st);
        ensure_keep(w->hscore, need * sizeof(int32_t), (size_t)nhits * sizeof(int32_t), st);
    }

    void run_batch(const std::vector<WorkItem> &items);
    void dna_level(int64_t &F, int cur, int64_t &cur_ent, int64_t &lf_ent_base, int64_t &lf_node_base,
                   int64_t &rh_base, const WorkItem *d_items);
    void run_batch_split(const std::vector<WorkItem> &items);
    void compact_hits(int64_t from);
    void leaf_phase(int64_t ninj);
    void locate_phase(int64_t nrh);
    int64_t finish(ae_hit **out_dev, std::vector<int64_t> &counts);
};

void Search::run_batch(const std::vector<WorkItem> &items) {
    int32_t batch_max_q = last_batch_q;
    for (const WorkItem &it : items) {
        if (it.c0 != 0 || it.c1 != m[it.qid] || it.qid <= last_batch_q) batches_ordered = false;
        batch_max_q = std::max(batch_max_q, it.qid);
    }
    const int sigma = ix.sigma;
    const int64_t batch_hits0 = nhits;
    const int nitems = (int)items.size();
    ensure(w->items, sizeof(WorkItem) * items.size(), st);
    CU(cudaMemcpyAsync(w->items.p, items.data(), sizeof(WorkItem) * items.size(), cudaMemcpyHostToDevice, st));
    const WorkItem *d_items = ptr<WorkItem>(w->items);
    auto t0 = std::chrono::steady_clock::now();
    batch_hint = -1;
    if (opt.hint_hits) {       // each query's hint, pro rata to its columns in this batch
        batch_hint = 0;
        for (const WorkItem &it : items)
            if (m[it.qid] > 0)
                batch_hint += (double)std::max<int64_t>(opt.hint_hits[it.qid], 0) * (double)(it.c1 - it.c0) /
                              (double)m[it.qid];
    }

    int cur = 0;
    int64_t F = 0;
    int depth = d0;
    // int16x2 rows while every live state fits: states at depth d are at most
    // d * g_max; past the limit the frontier is unpacked to int32 once
    bool i16 = opt.int16_limit > 0 && (int64_t)(d0 + 1) * sc.gmax <= opt.int16_limit;
    int64_t cur_ent = 0;
    if (d0 >= 1) {
        // ---- seed: (item, (d0)-gram) keys of every start column, sorted
        std::vector<int64_t> ipos(nitems + 1, 0);
        for (int i = 0; i < nitems; ++i) {
            const WorkItem &it = items[i];
            int64_t hi = std::min<int64_t>(it.c1, (int64_t)m[it.qid] - d0 + 1);
            ipos[i + 1] = ipos[i] + std::max<int64_t>(0, hi - it.c0);
        }
        const int64_t npos = ipos[nitems];
        if (npos == 0) return;
        ensure(w->item_pos, sizeof(int64_t) * ipos.size(), st);
        CU(cudaMemcpyAsync(w->item_pos.p, ipos.data(), sizeof(int64_t) * ipos.size(), cudaMemcpyHostToDevice, st));
        SeedArgs sa;
        sa.ix = ix;
        sa.sc = sc;
        sa.qv = qv;
        sa.items = d_items;
        sa.item_pos = ptr<int64_t>(w->item_pos);
        sa.nitems = nitems;
        sa.d0 = d0;
        sa.npos = npos;
        sa.int16 = i16 ? 1 : 0;
        // the domination table is allocated once per index (never from the static array)
        sa.dom = (opt.qprefix_domination && !g_arena) ? dom_table(idx, d0, st) : nullptr;
        sa.dominated = (unsigned long long *)((char *)w->stats.p + offsetof(DevStats, dominated));
        sa.parts = opt.fork_parts;
        sa.part = opt.fork_part;
        ensure(w->sk0, npos * 8, st);
        ensure(w->sv0, npos * 4, st);
        ensure(w->sk1, npos * 8, st);
        ensure(w->sv1, npos * 4, st);
        ensure(w->sort_tmp, ae_sort_tmp_words(npos) * 8, st);
        prof.mark(K_OTHER);
        ae_seed_keys(sa, ptr<uint64_t>(w->sk0), ptr<uint32_t>(w->sv0), st);
        prof.mark(K_OTHER);
        const int key_bits = (sigma == 4 ? 2 : 5) * d0 + bits_for(nitems);
        prof.mark(K_SORT);
        int which = ae_radix_sort(ptr<uint64_t>(w->sk0), ptr<uint32_t>(w->sv0), ptr<uint64_t>(w->sk1),
                                  ptr<uint32_t>(w->sv1), npos, key_bits, ptr<uint64_t>(w->sort_tmp), st);
        prof.mark(K_SORT);
        uint64_t *keys = which ? ptr<uint64_t>(w->sk1) : ptr<uint64_t>(w->sk0);
        uint32_t *vals = which ? ptr<uint32_t>(w->sv1) : ptr<uint32_t>(w->sv0);
        ensure(w->cnt[0], npos * 4, st);
        ensure(w->off[0], npos * 8, st);
        ensure(w->scan_tmp, ae_scan_tmp_words(npos, 5) * 8, st);
        ensure(w->totals, 64, st);
        ensure(w->nodes[cur], npos * sizeof(Node), st);
        ensure(w->aj[cur], npos * 4, st);
        ensure(w->aM[cur], npos * 4, st);
        ensure(w->aGa[cur], npos * 4, st);
        prof.mark(K_OTHER);
        ae_seed_nodes(sa, keys, vals, npos, key_bits, ptr<uint32_t>(w->cnt[0]), ptr<uint64_t>(w->off[0]),
                      ptr<uint64_t>(w->scan_tmp), ptr<Node>(w->nodes[cur]), ptr<int32_t>(w->aj[cur]),
                      ptr<int32_t>(w->aM[cur]), ptr<int32_t>(w->aGa[cur]), ptr<uint64_t>(w->totals), st);
        prof.mark(K_OTHER);
        CU(cudaMemcpyAsync(tot(), w->totals.p, 8, cudaMemcpyDeviceToHost, st));
        sync();
        F = (int64_t)tot()[0];
        cur_ent = npos;
    } else {
        // ---- root: one node per item with the implicit row M(0, j) = 0
        std::vector<Node> roots(nitems);
        for (int i = 0; i < nitems; ++i) {
            roots[i].lo = 0;
            roots[i].hi = (uint32_t)ix.rows;
            roots[i].item = i;
            roots[i].cnt = AE_ROOT_ROW;
            roots[i].off = 0;
        }
        ensure(w->nodes[cur], sizeof(Node) * nitems, st);
        CU(cudaMemcpyAsync(w->nodes[cur].p, roots.data(), sizeof(Node) * nitems, cudaMemcpyHostToDevice, st));
        for (int b = 0; b < 2; ++b) {
            ensure(w->aj[b], 256, st);
            ensure(w->aM[b], 256, st);
            ensure(w->aGa[b], 256, st);
        }
        F = nitems;
        sync();
    }

    // ---- trie levels
    int64_t lf_ent_base = 0, lf_node_base = 0, rh_base = 0;
    int64_t L_max_all = 0;
    dna_ratio_ok = false;   // the batch's first DNA level sizes its arenas from the first-level ratios
    for (int q = 0; q < nq; ++q) {
        int64_t Lm = std::max<int64_t>(m[q], m[q] + (int64_t)floor((double)(H[q] - ((int64_t)sc.sa * m[q] + sc.sg)) / sc.ss));
        L_max_all = std::max(L_max_all, Lm);
    }
    ensure(w->totals, 64, st);
    ensure(w->ctr, sizeof(LevelCounters), st);
    CU(cudaMemsetAsync(w->ctr.p, 0, sizeof(LevelCounters), st));   // clears the sticky overflow flag
    bool root_level = d0 < 1;   // the first level of a walk from the root has implicit rows
    while (F > 0 && depth <= L_max_all) {
        if (i16 && (int64_t)(depth + 1) * sc.gmax > opt.int16_limit) {
            ensure(w->aGa[cur], std::max<int64_t>(cur_ent, 1) * 4, st);
            prof.mark(K_OTHER);
            ae_mg_to_i32(ptr<int32_t>(w->aM[cur]), ptr<int32_t>(w->aGa[cur]), cur_ent, st);
            prof.mark(K_OTHER);
            i16 = false;
            ++stats.reroutes;
        }
        if (sigma == 4 && i16 && !opt.tier_stats && !root_level && !opt.general_rows && -sc.ss < 65536) {
            // DNA int16x2 route: one lane per parent entry, child ranges taken in
            // the task prologue (no separate children / compaction passes)
            dna_level(F, cur, cur_ent, lf_ent_base, lf_node_base, rh_base, d_items);
            cur ^= 1;
            ++depth;
            stats.levels++;
            stats.levels_int16++;
            continue;
        }
        root_level = false;
        // children per node (backward-search step per letter), scanned into
        // segment and triple offsets
        for (int k = 0; k < 2; ++k) {
            ensure(w->cnt[k], F * 4, st);
            ensure(w->off[k], F * 8, st);
        }
        ensure(w->scan_tmp, ae_scan_tmp_words(F, 5) * 8, st);
        ChildrenArgs ca;
        ca.ix = ix;
        ca.items = d_items;
        ca.nodes = ptr<Node>(w->nodes[cur]);
        ca.nnodes = F;
        ca.nseg = ptr<uint32_t>(w->cnt[0]);
        ca.ntrip = ptr<uint32_t>(w->cnt[1]);
        ca.stats = ptr<DevStats>(w->stats);
        prof.mark(K_EXPAND);
        ae_children(ca, st);
        const uint32_t *cin[2] = {ca.nseg, ca.ntrip};
        uint64_t *cout[2] = {ptr<uint64_t>(w->off[0]), ptr<uint64_t>(w->off[1])};
        ae_scan_u32(cin, cout, 2, F, ptr<uint64_t>(w->totals), ptr<uint64_t>(w->scan_tmp), st);
        prof.mark(K_EXPAND);
        CU(cudaMemcpyAsync(tot(), w->totals.p, 16, cudaMemcpyDeviceToHost, st));
        sync();
        const int64_t nseg = (int64_t)tot()[0], ntrip = (int64_t)tot()[1];
        stats.triples += ntrip;
        if (nseg == 0) break;
        ensure(w->segs, nseg * sizeof(Seg), st);
        ensure(w->seg_cnt, nseg * 4, st);
        ensure(w->seg_hit, nseg * 4, st);
        ensure(w->task_first, (ntrip / AE_ROW_TASK + 2) * 8, st);
        prof.mark(K_EXPAND);
        ae_compact_segs(ca, cout[0], cout[1], ptr<Seg>(w->segs), ptr<uint64_t>(w->task_first), st);
        prof.mark(K_EXPAND);
        const int nxt = cur ^ 1;
        RowsArgs ra;
        memset(&ra, 0, sizeof(ra));
        ra.ix = ix;
        ra.sc = sc;
        ra.qv = qv;
        ra.items = d_items;
        ra.nodes = ptr<Node>(w->nodes[cur]);
        ra.pj = ptr<int32_t>(w->aj[cur]);
        ra.pM = ptr<int32_t>(w->aM[cur]);
        ra.pGa = ptr<int32_t>(w->aGa[cur]);
        ra.segs = ptr<Seg>(w->segs);
        ra.nseg_dev = ptr<uint64_t>(w->totals);
        ra.ntrip_dev = ptr<uint64_t>(w->totals) + 1;
        ra.seg_cnt = ptr<uint32_t>(w->seg_cnt);
        ra.seg_hit = ptr<uint32_t>(w->seg_hit);
        ra.task_first = ptr<uint64_t>(w->task_first);
        ra.ctr = ptr<LevelCounters>(w->ctr);
        ra.stats = ptr<DevStats>(w->stats);
        ra.leaf_delay = opt.leaf_delay;
        ra.int16 = i16 ? 1 : 0;
        ra.tiers = opt.tier_stats ? 1 : 0;
        ra.parts = opt.fork_parts;
        ra.part = opt.fork_part;
        // count pass: exact output sizes of this level
        LevelCounters h0;
        memset(&h0, 0, sizeof(h0));
        h0.lf_ent = (unsigned long long)lf_ent_base;
        h0.lf_node = (unsigned long long)lf_node_base;
        h0.hits = (unsigned long long)rh_base;
        upload_level_counters(ptr<LevelCounters>(w->ctr), h0, st);
        const int64_t ntask = (ntrip + AE_ROW_TASK - 1) / AE_ROW_TASK;
        ensure(w->task_tot, (size_t)std::max<int64_t>(ntask, 1) * 5 * 4, st);
        ensure(w->task_off, (size_t)std::max<int64_t>(ntask, 1) * 5 * 8, st);
        ensure(w->task_tmp, (size_t)ae_scan_tmp_words(std::max<int64_t>(ntask, 1), 5) * 8, st);
        ensure(w->task_sum, 5 * 8, st);
        ra.task_tot = ptr<uint32_t>(w->task_tot);
        ra.task_stride = (uint64_t)ntask;
        ra.res = nullptr;
        ra.res_key = nullptr;
        if (i16 && !opt.tier_stats) {
            ensure(w->res, (size_t)std::max<int64_t>(ntrip, 1) * 4, st);
            ensure(w->res_key, (size_t)std::max<int64_t>(ntrip, 1) * 4, st);
            ra.res = ptr<uint32_t>(w->res);
            ra.res_key = ptr<int32_t>(w->res_key);
        }
        prof.mark(K_ROWS);
        ae_rows(ra, false, num_sms * ae_rows_blocks_per_sm(false), st);
        // write-pass bases: exclusive scan of the per-task output counts
        const uint32_t *tin[5];
        uint64_t *tout[5];
        for (int q = 0; q < 5; ++q) {
            tin[q] = ptr<uint32_t>(w->task_tot) + q * ntask;
            tout[q] = ptr<uint64_t>(w->task_off) + q * ntask;
        }
        ae_scan_u32(tin, tout, 5, ntask, ptr<uint64_t>(w->task_sum), ptr<uint64_t>(w->task_tmp), st);
        prof.mark(K_ROWS);
        LevelCounters hc;
        CU(cudaMemcpyAsync(tot(), w->ctr.p, sizeof(hc), cudaMemcpyDeviceToHost, st));
        sync();
        memcpy(&hc, tot(), sizeof(hc));
        if (hc.overflow) throw ae_error{AE_ECUDA};
        const int64_t fr_ent = (int64_t)hc.c_fr_ent, fr_node = (int64_t)hc.c_fr_node;
        const int64_t lf_ent = (int64_t)hc.c_lf_ent, lf_node = (int64_t)hc.c_lf_node, hits = (int64_t)hc.c_hits;
        ensure(w->aj[nxt], std::max<int64_t>(fr_ent, 1) * 4, st);
        ensure(w->aM[nxt], std::max<int64_t>(fr_ent, 1) * 4, st);
        if (!i16) ensure(w->aGa[nxt], std::max<int64_t>(fr_ent, 1) * 4, st);
        ensure(w->nodes[nxt], std::max<int64_t>(fr_node, 1) * sizeof(Node), st);
        ensure_keep(w->lj, (size_t)(lf_ent_base + lf_ent + 1) * 4, (size_t)lf_ent_base * 4, st);
        ensure_keep(w->lM, (size_t)(lf_ent_base + lf_ent + 1) * 4, (size_t)lf_ent_base * 4, st);
        ensure_keep(w->lGa, (size_t)(lf_ent_base + lf_ent + 1) * 4, (size_t)lf_ent_base * 4, st);
        ensure_keep(w->inj, (size_t)(lf_node_base + lf_node + 1) * sizeof(Inject),
                    (size_t)lf_node_base * sizeof(Inject), st);
        ensure_keep(w->rhits, (size_t)(rh_base + hits + 1) * sizeof(RangeHit), (size_t)rh_base * sizeof(RangeHit),
                    st);
        ra.fj = ptr<int32_t>(w->aj[nxt]);
        ra.fM = ptr<int32_t>(w->aM[nxt]);
        ra.fGa = ptr<int32_t>(w->aGa[nxt]);
        ra.fnodes = ptr<Node>(w->nodes[nxt]);
        ra.fr_ent_cap = (uint64_t)fr_ent;
        ra.fr_node_cap = (uint64_t)fr_node;
        ra.lj = ptr<int32_t>(w->lj);
        ra.lM = ptr<int32_t>(w->lM);
        ra.lGa = ptr<int32_t>(w->lGa);
        ra.inj = ptr<Inject>(w->inj);
        ra.lf_ent_cap = (uint64_t)(lf_ent_base + lf_ent);
        ra.lf_node_cap = (uint64_t)(lf_node_base + lf_node);
        ra.rhits = ptr<RangeHit>(w->rhits);
        ra.hit_cap = (uint64_t)(rh_base + hits);
        ra.stats = ptr<DevStats>(w->stats);
        ra.task_off = hc.wide ? nullptr : ptr<uint64_t>(w->task_off);
        ra.base_off[0] = 0;
        ra.base_off[1] = (uint64_t)lf_ent_base;
        ra.base_off[2] = 0;
        ra.base_off[3] = (uint64_t)lf_node_base;
        ra.base_off[4] = (uint64_t)rh_base;
        prof.mark(K_ROWS);
        ae_rows(ra, true, num_sms * ae_rows_blocks_per_sm(true), st);
        prof.mark(K_ROWS);
        if (trace())
            fprintf(stderr, "[ae level] depth %d nodes %lld segs %lld triples %lld -> frontier %lld nodes %lld, leaf %lld rows %lld\n",
                    depth, (long long)F, (long long)nseg, (long long)ntrip, (long long)fr_ent, (long long)fr_node,
                    (long long)lf_ent, (long long)lf_node);
        lf_ent_base += lf_ent;
        lf_node_base += lf_node;
        rh_base += hits;
        cur = nxt;
        F = fr_node;
        cur_ent = fr_ent;
        ++depth;
        stats.levels++;
        if (i16) stats.levels_int16++;
    }
    {
        LevelCounters hc;
        CU(cudaMemcpyAsync(tot(), w->ctr.p, sizeof(hc), cudaMemcpyDeviceToHost, st));
        sync();
        memcpy(&hc, tot(), sizeof(hc));
        if (hc.overflow) throw ae_error{AE_ECUDA};
    }
    CU(cudaGetLastError());
    sync();
    stats.ms_trie += ms_since(t0);
    stats.injections += lf_node_base;

    auto t1 = std::chrono::steady_clock::now();
    leaf_phase(lf_node_base);
    stats.ms_leaf += ms_since(t1);
    auto t2 = std::chrono::steady_clock::now();
    locate_phase(rh_base);
    compact_hits(batch_hits0);
    last_batch_q = batch_max_q;
    stats.ms_reduce += ms_since(t2);
}

// Row entries each lane of the DNA row kernel's walk layout can keep from its
// count phase for the write phase (per task)
#ifndef AE_STAGE_ROWS
#define AE_STAGE_ROWS 256
#endif

// Slots for sweep walks handed on to thread blocks (12 row buffers of the
// sweep's row capacity each; a walk that finds no free slot stays on its warp)
#ifndef AE_LEAF_WIDE_SLOTS
#define AE_LEAF_WIDE_SLOTS 512
#endif

// Levels of at most AE_WIDE_NODES nodes whose rows average AE_WIDE_ROW_AVG
// entries or more give each node a whole block (k_rows_dna_wide)
#ifndef AE_WIDE_NODES
#define AE_WIDE_NODES 65536
#endif
#ifndef AE_WIDE_ROW_AVG
#define AE_WIDE_ROW_AVG 512
#endif

// Average parent-row length up to which a level's rows are walked one lane per
// (node, child) rather than spread one entry per lane (per level on the 100 Mbp
// text with queries of 10 kbp to 1 Mbp, the walk was the faster layout up to
// rows of about 250 entries and the spread one from about 270)
#ifndef AE_SEQ_ROW_AVG
#define AE_SEQ_ROW_AVG 256
#endif

// One trie level of the DNA int16x2 route (ae_rows_dna.cu) in one launch.
// The output arenas are sized ahead from the previous level's output per input
// (with headroom); the kernel reserves every task's ranges on the level
// cursors, which end at the level's exact totals.  If a reservation passed a
// capacity the arenas are grown to those totals and the level is run again.
// Nodes and arenas have the layout of the general route.
void Search::dna_level(int64_t &F, int cur, int64_t &cur_ent, int64_t &lf_ent_base, int64_t &lf_node_base,
                       int64_t &rh_base, const WorkItem *d_items) {
    (void)d_items;
    const int nxt = cur ^ 1;
    // nodes per task: 32 (one per lane) unless the level is too small to give
    // every resident warp a few tasks
    const int64_t warps = (int64_t)num_sms * ae_rows_dna_blocks_per_sm() * ae_rows_dna_warps_per_block();
    const int npt = (int)std::max<int64_t>(1, std::min<int64_t>(32, F / (warps * 4)));

    // expected outputs: per kind (frontier entries, leaf entries, frontier
    // nodes, leaf nodes, hits) the previous level's ratio to its input, plus a
    // fifth; the first level of a batch assumes four children per node
    static const double first_ratio[5] = {8.0, 1.0, 4.0, 1.0, 0.25};
    const double in[5] = {(double)cur_ent, (double)cur_ent, (double)F, (double)F, (double)cur_ent};
    int64_t want[5];
    for (int q = 0; q < 5; ++q) {
        double r = dna_ratio_ok ? dna_ratio[q] * 1.2 : first_ratio[q];
        // a large level's output is guessed at most 1.5 times its input: the growth
        // ratio peaks and falls within a few levels, and sizing every later level by
        // the peak ratio would hold several times the memory the search needs (a
        // short guess costs one more run of the level, and only until the buffers
        // have grown)
        if (r * in[q] > (double)(1 << 28)) r = std::min(r, 1.5);
        want[q] = (int64_t)(r * in[q]) + 256;
    }
    want[2] = std::min<int64_t>(want[2], 4 * F);   // a node has at most four children
    want[3] = std::min<int64_t>(want[3], 4 * F);
    // grow ahead only outside the fixed arena, and only as far as memory allows:
    // a capacity that falls short costs one more run of the level
    auto grow = [&](int64_t fe, int64_t le, int64_t fn, int64_t ln, int64_t h, bool exact) {
        auto one = [&](auto fn_) {
            if (exact) {
                fn_();
                return;
            }
            if (g_arena) return;
            try {
                fn_();
            } catch (const ae_error &e) {
                if (e.st != AE_ENOMEM) throw;
            }
        };
        one([&] { ensure(w->aj[nxt], (size_t)std::max<int64_t>(fe, 1) * 4, st); });
        one([&] { ensure(w->aM[nxt], (size_t)std::max<int64_t>(fe, 1) * 4, st); });
        one([&] { ensure(w->nodes[nxt], (size_t)std::max<int64_t>(fn, 1) * sizeof(Node), st); });
        one([&] { ensure_keep(w->lj, (size_t)(lf_ent_base + le + 1) * 4, (size_t)lf_ent_base * 4, st); });
        one([&] { ensure_keep(w->lM, (size_t)(lf_ent_base + le + 1) * 4, (size_t)lf_ent_base * 4, st); });
        one([&] { ensure_keep(w->lGa, (size_t)(lf_ent_base + le + 1) * 4, (size_t)lf_ent_base * 4, st); });
        one([&] {
            ensure_keep(w->inj, (size_t)(lf_node_base + ln + 1) * sizeof(Inject), (size_t)lf_node_base * sizeof(Inject),
                        st);
        });
        one([&] {
            ensure_keep(w->rhits, (size_t)(rh_base + h + 1) * sizeof(RangeHit), (size_t)rh_base * sizeof(RangeHit),
                        st);
        });
    };
    grow(want[0], want[1], want[2], want[3], want[4], false);

    DnaRowsArgs da;
    memset(&da, 0, sizeof(da));
    da.ix = ix;
    da.sc = sc;
    da.qv = qv;
    da.nnodes = F;
    da.nodes_per_task = npt;
    da.leaf_delay = opt.leaf_delay;
    {
        const uint64_t u = (uint64_t)(-(int64_t)sc.ss);
        da.urec = ((1ull << 32) + u - 1) / u;
    }
    // short parent rows are walked one lane per (node, child); long rows spread
    // over the lanes (a lone long row would hold its warp alone)
    da.sequential = (opt.row_layout == 1) || (opt.row_layout == 0 && cur_ent <= AE_SEQ_ROW_AVG * F) ? 1 : 0;
    // a level of few nodes with long rows: one block per node
    if (opt.row_layout == 3 || (opt.row_layout == 0 && F <= AE_WIDE_NODES && cur_ent >= AE_WIDE_ROW_AVG * F))
        da.sequential = 2;
    // the walk layout keeps its count phase's rows for the write phase (outside the
    // fixed arena of the no-allocation entry point; without room, rows are computed twice)
    da.stage = nullptr;
    da.stage_cap = 0;
    if (da.sequential == 1 && !g_arena) {
        const int64_t lanes = (int64_t)num_sms * ae_rows_dna_blocks_per_sm() * ae_rows_dna_warps_per_block() * 32;
        try {
            ensure(w->stage, (size_t)lanes * AE_STAGE_ROWS * sizeof(uint2), st);
            da.stage = ptr<uint2>(w->stage);
            da.stage_cap = AE_STAGE_ROWS;
        } catch (const ae_error &e) {
            if (e.st != AE_ENOMEM) throw;
        }
    }
    const auto t_level = std::chrono::steady_clock::now();
    LevelCounters hc;
    auto run = [&]() {
        LevelCounters h0;
        memset(&h0, 0, sizeof(h0));
        h0.lf_ent = (unsigned long long)lf_ent_base;
        h0.lf_node = (unsigned long long)lf_node_base;
        h0.hits = (unsigned long long)rh_base;
        upload_level_counters(ptr<LevelCounters>(w->ctr), h0, st);
        // capacities are the buffers' sizes (the leaf and hit arenas keep one spare slot)
        auto cap = [](const DevBuf &b, size_t elem, int64_t spare) {
            return (uint64_t)std::max<int64_t>((int64_t)(b.bytes / elem) - spare, 0);
        };
        da.nodes = ptr<Node>(w->nodes[cur]);
        da.pj = ptr<int32_t>(w->aj[cur]);
        da.pmg = ptr<uint32_t>(w->aM[cur]);
        da.fj = ptr<int32_t>(w->aj[nxt]);
        da.fmg = ptr<uint32_t>(w->aM[nxt]);
        da.fnodes = ptr<Node>(w->nodes[nxt]);
        da.fr_ent_cap = std::min(cap(w->aj[nxt], 4, 0), cap(w->aM[nxt], 4, 0));
        da.fr_node_cap = cap(w->nodes[nxt], sizeof(Node), 0);
        da.lj = ptr<int32_t>(w->lj);
        da.lM = ptr<int32_t>(w->lM);
        da.lGa = ptr<int32_t>(w->lGa);
        da.inj = ptr<Inject>(w->inj);
        da.lf_ent_cap = std::min({cap(w->lj, 4, 1), cap(w->lM, 4, 1), cap(w->lGa, 4, 1)});
        da.lf_node_cap = cap(w->inj, sizeof(Inject), 1);
        da.rhits = ptr<RangeHit>(w->rhits);
        da.hit_cap = cap(w->rhits, sizeof(RangeHit), 1);
        da.ctr = ptr<LevelCounters>(w->ctr);
        prof.mark(K_ROWS);
        ae_rows_dna(da, num_sms * ae_rows_dna_blocks_per_sm(), st);
        prof.mark(K_ROWS);
        CU(cudaMemcpyAsync(tot(), w->ctr.p, sizeof(hc), cudaMemcpyDeviceToHost, st));
        sync();
        memcpy(&hc, tot(), sizeof(hc));
        if (hc.overflow) throw ae_error{AE_ECUDA};   // the two phases of a task disagreed
    };
    run();
    int64_t fr_ent = (int64_t)hc.fr_ent, fr_node = (int64_t)hc.fr_node;
    int64_t lf_ent = (int64_t)hc.lf_ent - lf_ent_base, lf_node = (int64_t)hc.lf_node - lf_node_base;
    int64_t hits = (int64_t)hc.hits - rh_base;
    const bool retried = hc.retry != 0;
    if (retried) {
        ++dna_retries;
        grow(fr_ent, lf_ent, fr_node, lf_node, hits, true);
        run();
        if (hc.retry || (int64_t)hc.fr_ent != fr_ent || (int64_t)hc.fr_node != fr_node ||
            (int64_t)hc.lf_ent - lf_ent_base != lf_ent || (int64_t)hc.lf_node - lf_node_base != lf_node ||
            (int64_t)hc.hits - rh_base != hits)
            throw ae_error{AE_ECUDA};   // the same level gave other totals
    }
    stats.triples += (int64_t)hc.triples;
    dna_nodes += F;
    dna_entries += fr_ent + lf_ent;
    {
        const double out[5] = {(double)fr_ent, (double)lf_ent, (double)fr_node, (double)lf_node, (double)hits};
        for (int q = 0; q < 5; ++q) dna_ratio[q] = in[q] > 0 ? out[q] / in[q] : 0.0;
        dna_ratio_ok = true;
    }
    if (trace()) {
        fprintf(stderr, "[ae level] dna %s nodes %lld (per task %d) entries %lld triples %lld -> frontier %lld nodes %lld, "
                        "leaf %lld rows %lld%s; %.3f ms\n",
                da.sequential == 2 ? "block" : da.sequential ? "walk" : "spread", (long long)F, npt, (long long)cur_ent,
                (long long)hc.triples,
                (long long)fr_ent, (long long)fr_node, (long long)lf_ent, (long long)lf_node,
                retried ? " (run again at exact sizes)" : "", ms_since(t_level));
    }
    lf_ent_base += lf_ent;
    lf_node_base += lf_node;
    rh_base += hits;
    F = fr_node;
    cur_ent = fr_ent;
}

// Reduce the hits [from, nhits) of the batch just finished to one record per
// (query, text end, query end) with the maximum score, in place.  Queries are
// whole inside a batch by default, so the final pass then sorts far fewer
// records; it stays exact either way.
// A batch whose working set does not fit the device is split in two and each
// half searched alone (batches are independent: a work item's forks start in
// its own columns, and hits meet only at the final per-cell maximum).  The
// failed attempt's hits are dropped; its counters stay in the statistics.
void Search::run_batch_split(const std::vector<WorkItem> &items) {
    const int64_t h0 = nhits;
    try {
        run_batch(items);
        return;
    } catch (const ae_error &e) {
        if (e.st != AE_ENOMEM) throw;
    }
    cudaGetLastError();
    CU(cudaStreamSynchronize(st));
    nhits = h0;
    ++stats.batch_splits;
    if (!g_arena) w->trim_batch();
    std::vector<WorkItem> a, b;
    if (items.size() >= 2) {
        a.assign(items.begin(), items.begin() + (long)(items.size() / 2));
        b.assign(items.begin() + (long)(items.size() / 2), items.end());
    } else {
        const WorkItem it = items[0];
        if (it.c1 - it.c0 < 2) throw ae_error{AE_ENOMEM};
        const int32_t mid = it.c0 + (it.c1 - it.c0) / 2;
        WorkItem x = it, y = it;
        x.c1 = mid;
        y.c0 = mid;
        a.push_back(x);
        b.push_back(y);
    }
    run_batch_split(a);
    run_batch_split(b);
}

void Search::compact_hits(int64_t from) {
    const int64_t N = nhits - from;
    if (N <= 1) return;
    ensure(w->hk1, N * 8, st);
    ensure(w->hv1, N * 4, st);
    ensure(w->sort_tmp, ae_sort_tmp_words(N) * 8, st);
    uint64_t *k0 = ptr<uint64_t>(w->hkey) + from;
    uint32_t *v0 = reinterpret_cast<uint32_t *>(ptr<int32_t>(w->hscore) + from);
    prof.mark(K_SORT);
    int which = ae_radix_sort(k0, v0, ptr<uint64_t>(w->hk1), ptr<uint32_t>(w->hv1), N, be + bj + bq,
                              ptr<uint64_t>(w->sort_tmp), st);
    prof.mark(K_SORT);
    const uint64_t *keys = which ? ptr<uint64_t>(w->hk1) : k0;
    const int32_t *scores = which ? ptr<int32_t>(w->hv1) : reinterpret_cast<int32_t *>(v0);
    ensure(w->uflags, N * 4, st);
    ensure(w->uoff, N * 8, st);
    ensure(w->scan_tmp, ae_scan_tmp_words(N, 5) * 8, st);
    prof.mark(K_OTHER);
    ae_unique_flags(keys, N, ptr<uint32_t>(w->uflags), st);
    const uint32_t *in[1] = {ptr<uint32_t>(w->uflags)};
    uint64_t *out[1] = {ptr<uint64_t>(w->uoff)};
    ae_scan_u32(in, out, 1, N, ptr<uint64_t>(w->totals), ptr<uint64_t>(w->scan_tmp), st);
    CU(cudaMemcpyAsync(tot(), w->totals.p, 8, cudaMemcpyDeviceToHost, st));
    sync();
    const int64_t U = (int64_t)tot()[0];
    // compacted records go to the other buffer, then back in place
    uint64_t *dk = which ? k0 : ptr<uint64_t>(w->hk1);
    int32_t *ds = which ? reinterpret_cast<int32_t *>(v0) : ptr<int32_t>(w->hv1);
    ae_unique_compact(keys, scores, N, ptr<uint64_t>(w->uoff), dk, ds, st);
    if (!which) {
        CU(cudaMemcpyAsync(k0, dk, U * 8, cudaMemcpyDeviceToDevice, st));
        CU(cudaMemcpyAsync(v0, ds, U * 4, cudaMemcpyDeviceToDevice, st));
    }
    prof.mark(K_OTHER);
    if (trace()) fprintf(stderr, "[ae hits] batch raw %lld -> unique %lld\n", (long long)N, (long long)U);
    nhits = from + U;
}

void Search::leaf_phase(int64_t ninj) {
    if (ninj <= 0) return;
    ensure(w->sk0, ninj * 8, st);
    ensure(w->sv0, ninj * 4, st);
    ensure(w->sk1, ninj * 8, st);
    ensure(w->sv1, ninj * 4, st);
    ensure(w->sort_tmp, ae_sort_tmp_words(ninj) * 8, st);
    prof.mark(K_SORT);
    ae_inject_keys(ptr<Inject>(w->inj), ninj, ptr<uint64_t>(w->sk0), ptr<uint32_t>(w->sv0), st);
    int which = ae_radix_sort(ptr<uint64_t>(w->sk0), ptr<uint32_t>(w->sv0), ptr<uint64_t>(w->sk1),
                              ptr<uint32_t>(w->sv1), ninj, 32 + bits_for(std::max(nq - 1, 1)),
                              ptr<uint64_t>(w->sort_tmp), st);
    prof.mark(K_SORT);
    const uint32_t *order = which ? ptr<uint32_t>(w->sv1) : ptr<uint32_t>(w->sv0);

    const int threads = 128;
    const int blocks = num_sms * (g_arena ? 2 : 12);
    const int nwarps = blocks * threads / 32;
    if (w->leaf_cap < opt.leaf_capacity) w->leaf_cap = opt.leaf_capacity;
    ensure(w->next_seg, 8, st);
    ensure(w->hcount, 8, st);
    int64_t hit_cap = std::max<int64_t>(1 << 20, batch_hint >= 0 ? (int64_t)(1.25 * batch_hint) + 65536
                                                                 : (int64_t)(ninj * w->hit_ratio) + 4096);
    // wide walks move to blocks (not inside the fixed arena of the no-allocation
    // entry point, nor when entries are counted by tier, which only the warp walk does)
    const int32_t esc_min = (g_arena || opt.tier_stats) ? 0 : opt.leaf_wide_rows;
    const int32_t esc_max = esc_min > 0 ? AE_LEAF_WIDE_SLOTS : 0;
    for (int attempt = 0; attempt < 12; ++attempt) {
        ensure(w->scratch, (size_t)ae_leaf_scratch_words(w->leaf_cap, nwarps) * 4, st);
        if (esc_max > 0) {
            ensure(w->esc, (size_t)esc_max * sizeof(EscWalk), st);
            ensure(w->esc_count, 8, st);
            ensure(w->esc_rows, (size_t)esc_max * 12 * (size_t)w->leaf_cap * 4, st);
            CU(cudaMemsetAsync(w->esc_count.p, 0, 8, st));
        }
        hits_reserve(hit_cap);
        CU(cudaMemsetAsync(w->next_seg.p, 0, 8, st));
        unsigned long long base = (unsigned long long)nhits;
        CU(cudaMemcpyAsync(w->hcount.p, &base, 8, cudaMemcpyHostToDevice, st));
        CU(cudaMemsetAsync((char *)w->stats.p + offsetof(DevStats, leaf_overflow), 0, 16, st));
        LeafArgs la;
        memset(&la, 0, sizeof(la));
        la.ix = ix;
        la.sc = sc;
        la.qv = qv;
        la.inj = ptr<Inject>(w->inj);
        la.order = order;
        la.ninj = ninj;
        la.lj = ptr<int32_t>(w->lj);
        la.lM = ptr<int32_t>(w->lM);
        la.lGa = ptr<int32_t>(w->lGa);
        // injections per sweep task: the option, or (0 = auto) enough for about
        // eight tasks per warp -- longer tasks merge more rows that meet inside
        // homologous regions, fewer tasks balance worse
        la.seg = opt.leaf_segment > 0
                     ? opt.leaf_segment
                     : (int32_t)std::min<int64_t>(4096, std::max<int64_t>(32, ninj / ((int64_t)nwarps * 8)));
        la.nseg = (ninj + la.seg - 1) / la.seg;
        la.next_seg = ptr<unsigned long long>(w->next_seg);
        la.scratch = ptr<int32_t>(w->scratch);
        la.cap = w->leaf_cap;
        la.nwarps = nwarps;
        la.hit_key = ptr<uint64_t>(w->hkey);
        la.hit_score = ptr<int32_t>(w->hscore);
        la.hit_count = ptr<unsigned long long>(w->hcount);
        la.hit_cap = (uint64_t)(nhits + hit_cap);
        la.be = be;
        la.bj = bj;
        la.tiers = opt.tier_stats ? 1 : 0;
        la.stats = ptr<DevStats>(w->stats);
        la.esc_min = esc_max > 0 ? esc_min : 0;
        la.esc_max = esc_max;
        if (esc_max > 0) {
            la.esc_count = ptr<unsigned long long>(w->esc_count);
            la.esc = ptr<EscWalk>(w->esc);
            la.esc_rows = ptr<int32_t>(w->esc_rows);
        }
        prof.mark(K_LEAF);
        ++stats.leaf_sweeps;
        const auto t_sweep = std::chrono::steady_clock::now();
        ae_leaf_sweep(la, blocks, threads, st);
        prof.mark(K_LEAF);
        CU(cudaGetLastError());
        unsigned long long hdr[4] = {0, 0, 0, 0};
        CU(cudaMemcpyAsync(tot(), w->hcount.p, 8, cudaMemcpyDeviceToHost, st));
        CU(cudaMemcpyAsync(tot() + 1, (char *)w->stats.p + offsetof(DevStats, leaf_overflow), 16,
                           cudaMemcpyDeviceToHost, st));
        if (esc_max > 0) CU(cudaMemcpyAsync(tot() + 3, w->esc_count.p, 8, cudaMemcpyDeviceToHost, st));
        sync();
        hdr[0] = tot()[0];
        hdr[1] = tot()[1];
        hdr[2] = tot()[2];
        if (esc_max > 0) hdr[3] = std::min<unsigned long long>(tot()[3], (unsigned long long)esc_max);
        if (trace())
            fprintf(stderr, "[ae leaf] injections %lld (tasks %lld of %d) attempt %d: %.2f ms, hits %llu (cap %lld), row overflow %llu, hit overflow %llu, cap %d\n",
                    (long long)ninj, (long long)la.nseg, la.seg, attempt, ms_since(t_sweep),
                    hdr[0] - (unsigned long long)nhits, (long long)hit_cap, hdr[1], hdr[2], w->leaf_cap);
        if (hdr[1] != 0) {          // a row outgrew the scratch: retry larger
            // a sweep row holds at most two entries per query column plus gap runs, so
            // a capacity past 2^28 entries means something else is wrong: stop
            if (w->leaf_cap >= (1 << 28)) throw ae_error{AE_ENOMEM};
            w->leaf_cap *= 4;
            // the no-allocation entry point caps sweep rows at its documented limit
            if (g_arena && w->leaf_cap > AE_STATIC_MAX_LEAF_CAP) throw ae_error{AE_EUNSUPPORTED};
            continue;
        }
        if (hdr[2] != 0 || (int64_t)hdr[0] > nhits + hit_cap) {   // hit buffer too small
            hit_cap = (int64_t)hdr[0] - nhits + 1024;
            continue;
        }
        // hit records per injection vary by batch (homologous queries write many
        // more): keep the largest ratio seen, so a workspace sizes for its worst
        // batch instead of rerunning the sweep
        w->hit_ratio = std::max(w->hit_ratio,
                                std::min(64.0, 1.3 * (double)((int64_t)hdr[0] - nhits) / (double)ninj + 0.01));
        stats.leaf_raw_hits += (int64_t)hdr[0] - nhits;
        stats.leaf_wide_walks += (int64_t)hdr[3];
        nhits = (int64_t)hdr[0];
        return;
    }
    throw ae_error{AE_ENOMEM};
}

void Search::locate_phase(int64_t nrh) {
    if (nrh <= 0) return;
    ensure(w->cnt[0], nrh * 4, st);
    ensure(w->off[0], nrh * 8, st);
    ensure(w->scan_tmp, ae_scan_tmp_words(nrh, 5) * 8, st);
    prof.mark(K_OTHER);
    ae_locate_counts(ptr<RangeHit>(w->rhits), nrh, ptr<uint32_t>(w->cnt[0]), st);
    const uint32_t *in[1] = {ptr<uint32_t>(w->cnt[0])};
    uint64_t *out[1] = {ptr<uint64_t>(w->off[0])};
    ae_scan_u32(in, out, 1, nrh, ptr<uint64_t>(w->totals), ptr<uint64_t>(w->scan_tmp), st);
    prof.mark(K_OTHER);
    CU(cudaMemcpyAsync(tot(), w->totals.p, 8, cudaMemcpyDeviceToHost, st));
    sync();
    const int64_t total = (int64_t)tot()[0];
    hits_reserve(total);
    prof.mark(K_OTHER);
    ae_locate(ptr<RangeHit>(w->rhits), nrh, ptr<uint64_t>(w->off[0]), total, ix.tend, be, bj,
              ptr<uint64_t>(w->hkey) + nhits, ptr<int32_t>(w->hscore) + nhits, st);
    prof.mark(K_OTHER);
    nhits += total;
}

// Sort all point hits by (query, text end, query end) and keep the maximum
// score of each cell.  Returns the number of distinct results; *out_dev points
// into the workspace.
int64_t Search::finish(ae_hit **out_dev, std::vector<int64_t> &counts) {
    auto t0 = std::chrono::steady_clock::now();
    const int64_t N = nhits;
    counts.assign(nq, 0);
    ensure(w->qcount, sizeof(unsigned long long) * nq, st);
    CU(cudaMemsetAsync(w->qcount.p, 0, sizeof(unsigned long long) * nq, st));
    stats.raw_hits = N;
    if (N == 0) {
        *out_dev = nullptr;
        stats.ms_reduce += ms_since(t0);
        return 0;
    }
    if (batches_ordered) {
        // each batch's hits are sorted and unique, and the batches follow each other in
        // query order: the records are final as they lie
        ensure(w->uniq, std::max<int64_t>(N, 1) * sizeof(ae_hit), st);
        prof.mark(K_OTHER);
        ae_unique_write(ptr<uint64_t>(w->hkey), ptr<int32_t>(w->hscore), N, nullptr, be, bj, ptr<ae_hit>(w->uniq),
                        ptr<unsigned long long>(w->qcount), st);
        prof.mark(K_OTHER);
        std::vector<unsigned long long> qc(nq);
        CU(cudaMemcpyAsync(qc.data(), w->qcount.p, sizeof(unsigned long long) * nq, cudaMemcpyDeviceToHost, st));
        sync();
        for (int q = 0; q < nq; ++q) counts[q] = (int64_t)qc[q];
        *out_dev = ptr<ae_hit>(w->uniq);
        stats.hits = N;
        stats.ms_reduce += ms_since(t0);
        return N;
    }
    ensure(w->hk1, N * 8, st);
    ensure(w->hv1, N * 4, st);
    ensure(w->sort_tmp, ae_sort_tmp_words(N) * 8, st);
    prof.mark(K_SORT);
    int which = ae_radix_sort(ptr<uint64_t>(w->hkey), reinterpret_cast<uint32_t *>(w->hscore.p),
                              ptr<uint64_t>(w->hk1), ptr<uint32_t>(w->hv1), N, be + bj + bq,
                              ptr<uint64_t>(w->sort_tmp), st);
    prof.mark(K_SORT);
    const uint64_t *keys = which ? ptr<uint64_t>(w->hk1) : ptr<uint64_t>(w->hkey);
    const int32_t *scores = which ? ptr<int32_t>(w->hv1) : ptr<int32_t>(w->hscore);
    ensure(w->uflags, N * 4, st);
    ensure(w->uoff, N * 8, st);
    ensure(w->scan_tmp, ae_scan_tmp_words(N, 5) * 8, st);
    prof.mark(K_OTHER);
    ae_unique_flags(keys, N, ptr<uint32_t>(w->uflags), st);
    const uint32_t *in[1] = {ptr<uint32_t>(w->uflags)};
    uint64_t *out[1] = {ptr<uint64_t>(w->uoff)};
    ae_scan_u32(in, out, 1, N, ptr<uint64_t>(w->totals), ptr<uint64_t>(w->scan_tmp), st);
    prof.mark(K_OTHER);
    CU(cudaMemcpyAsync(tot(), w->totals.p, 8, cudaMemcpyDeviceToHost, st));
    sync();
    const int64_t U = (int64_t)tot()[0];
    ensure(w->uniq, std::max<int64_t>(U, 1) * sizeof(ae_hit), st);
    prof.mark(K_OTHER);
    ae_unique_write(keys, scores, N, ptr<uint64_t>(w->uoff), be, bj, ptr<ae_hit>(w->uniq),
                    ptr<unsigned long long>(w->qcount), st);
    prof.mark(K_OTHER);
    std::vector<unsigned long long> qc(nq);
    CU(cudaMemcpyAsync(qc.data(), w->qcount.p, sizeof(unsigned long long) * nq, cudaMemcpyDeviceToHost, st));
    sync();
    for (int q = 0; q < nq; ++q) counts[q] = (int64_t)qc[q];
    *out_dev = ptr<ae_hit>(w->uniq);
    stats.hits = U;
    stats.ms_reduce += ms_since(t0);
    return U;
}

// Shared core: codes already on the device in w->codes.
ae_status search_core(const ae_index *idx, Workspace *w, const int64_t *offsets, int32_t nq,
                      const ae_scoring *scoring, const int32_t *H, const ae_options *opt, cudaStream_t st,
                      ae_hit **out_dev, std::vector<int64_t> &counts, int64_t *total) {
    auto t0 = std::chrono::steady_clock::now();
    Search s;
    s.idx = idx;
    s.w = w;
    s.st = st;
    s.ix = idx->view;
    s.nq = nq;
    memset(&s.stats, 0, sizeof(s.stats));
    ae_options_default(&s.opt);
    if (opt) s.opt = *opt;
    if (s.opt.fork_parts < 1 || s.opt.fork_part < 0 || s.opt.fork_part >= s.opt.fork_parts) return AE_EINVAL;
    if (s.opt.leaf_wide_rows < 0) return AE_EINVAL;
    if (s.opt.row_layout < 0 || s.opt.row_layout > 3) return AE_EINVAL;
    if (s.opt.item_columns < 1 || s.opt.batch_columns < 1 || s.opt.leaf_capacity < 64 || s.opt.leaf_segment < 0 ||
        s.opt.leaf_delay < 0 || s.opt.leaf_delay > 14 || s.opt.int16_limit < 0 || s.opt.int16_limit > 32000)
        return AE_EINVAL;
    ae_status e = make_score(scoring, s.ix.sigma, s.sc);
    if (e != AE_OK) return e;
    s.off.assign(offsets, offsets + nq + 1);
    s.m.resize(nq);
    s.H.resize(nq);
    int32_t mmax = 1, Hmin = INT32_MAX;
    for (int q = 0; q < nq; ++q) {
        int64_t len = offsets[q + 1] - offsets[q];
        if (len < 0 || len >= (1 << 28) || H[q] < 1) return AE_EINVAL;
        s.m[q] = (int32_t)len;
        // no score reaches 2^30 (m * g_max < 2^30 is checked below), so a larger
        // threshold selects the same (empty) set and keeps device arithmetic in int32
        s.H[q] = std::min<int32_t>(H[q], 1 << 30);
        mmax = std::max(mmax, (int32_t)len);
        Hmin = std::min(Hmin, s.H[q]);
    }
    // keys of the max-plus scan stay within int32
    if ((int64_t)mmax * (-(int64_t)s.sc.ss + s.sc.gmax + 1) >= (1ll << 30)) return AE_EUNSUPPORTED;
    if (nq >= (1 << 24)) return AE_EUNSUPPORTED;
    s.be = bits_for(std::max<int64_t>(s.ix.n - 1, 1));
    s.bj = bits_for(std::max(mmax - 1, 1));
    s.bq = bits_for(std::max(nq - 1, 1));
    if (s.be + s.bj + s.bq > 64 || s.be > 32) return AE_EUNSUPPORTED;
    s.d0 = seed_depth(s.sc, Hmin, s.opt.qprefix_seed != 0);
    s.stats.seed_depth = s.d0;
    s.prof.on = s.opt.profile != 0;
    if (s.opt.workspace_limit < 0) return AE_EINVAL;
    g_cur_ws = w;
    g_ws_limit = g_arena ? 0 : s.opt.workspace_limit;
    struct LimitReset {
        ~LimitReset() {
            g_cur_ws = nullptr;
            g_ws_limit = 0;
        }
    } limit_reset;
    s.prof.st = st;
    const int64_t launches0 = ae_launches_read();
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&s.num_sms, cudaDevAttrMultiProcessorCount, dev);

    try {
        ensure(w->qoff, sizeof(int64_t) * (nq + 1), st);
        ensure(w->qm, sizeof(int32_t) * nq, st);
        ensure(w->qH, sizeof(int32_t) * nq, st);
        ensure(w->stats, sizeof(DevStats), st);
        CU(cudaMemcpyAsync(w->qoff.p, s.off.data(), sizeof(int64_t) * (nq + 1), cudaMemcpyHostToDevice, st));
        CU(cudaMemcpyAsync(w->qm.p, s.m.data(), sizeof(int32_t) * nq, cudaMemcpyHostToDevice, st));
        CU(cudaMemcpyAsync(w->qH.p, s.H.data(), sizeof(int32_t) * nq, cudaMemcpyHostToDevice, st));
        CU(cudaMemsetAsync(w->stats.p, 0, sizeof(DevStats), st));
        s.qv.codes = ptr<uint8_t>(w->codes);
        s.qv.off = ptr<int64_t>(w->qoff);
        s.qv.m = ptr<int32_t>(w->qm);
        s.qv.H = ptr<int32_t>(w->qH);

        // work items: columns of each query in slices of item_columns
        std::vector<WorkItem> batch;
        int64_t cols = 0;
        for (int q = 0; q < nq; ++q) {
            for (int64_t c0 = 0; c0 < s.m[q]; c0 += s.opt.item_columns) {
                WorkItem it;
                it.qid = q;
                it.c0 = (int32_t)c0;
                it.c1 = (int32_t)std::min<int64_t>(s.m[q], c0 + s.opt.item_columns);
                it.pad = 0;
                batch.push_back(it);
                cols += it.c1 - it.c0;
                if (cols >= s.opt.batch_columns) {
                    s.run_batch_split(batch);
                    batch.clear();
                    cols = 0;
                }
            }
        }
        if (!batch.empty()) s.run_batch_split(batch);
        *total = s.finish(out_dev, counts);
        DevStats ds;
        CU(cudaMemcpyAsync(&ds, w->stats.p, sizeof(ds), cudaMemcpyDeviceToHost, st));
        CU(cudaStreamSynchronize(st));
        s.stats.nodes = (int64_t)ds.nodes + s.dna_nodes;
        s.stats.leaf_rows = (int64_t)ds.leaf_rows;
        s.stats.entries = (int64_t)ds.entries + s.dna_entries;
        for (int k = 0; k < 3; ++k) s.stats.entries_tier[k] = (int64_t)ds.tier[k];
        s.stats.entries_leaf = (int64_t)ds.entries_leaf;
        s.stats.dominated = (int64_t)ds.dominated;
        s.stats.reused = (int64_t)ds.reused;
        s.stats.candidates = (int64_t)ds.cand;
        s.stats.pruned_nonpos = (int64_t)ds.pruned_nonpos;
        s.stats.pruned_reach = (int64_t)ds.pruned_reach;
        s.stats.leaf_max_steps = (int64_t)ds.leaf_max_steps;
        s.stats.leaf_max_width = (int64_t)ds.leaf_max_width;
        if (trace())
            fprintf(stderr, "[ae leaf] longest sweep task %.2f Mcycles (%.2f ms at 2.07 GHz)\n",
                    ds.leaf_max_cycles / 1e6, ds.leaf_max_cycles / 2.07e6);
        s.stats.ws_bytes = g_ws_bytes;
        s.stats.ms_k_expand = s.prof.ms(K_EXPAND);
        s.stats.ms_k_rows = s.prof.ms(K_ROWS);
        s.stats.ms_k_leaf = s.prof.ms(K_LEAF);
        s.stats.ms_k_sort = s.prof.ms(K_SORT);
        s.stats.ms_k_other = s.prof.ms(K_OTHER);
    } catch (const ae_error &err) {
        cudaGetLastError();
        return err.st;
    } catch (const std::bad_alloc &) {
        return AE_ENOMEM;
    }
    s.stats.ms_total = ms_since(t0);
    s.stats.launches = ae_launches_read() - launches0;
    g_last_stats = s.stats;
    return AE_OK;
}

}  // namespace

// ------------------------------------------------------------------ C ABI

namespace {

// Section 5 (1)-(2): the suffix array of the reversed text on the device
// (prefix doubling), the occurrence blocks and text-end array filled from it
// on the host, then the upload.
ae_status build_index(ae_index *idx, const uint8_t *codes, int64_t n, int32_t alphabet,
                      const int64_t *starts = nullptr, int32_t nseq = 0) {
    // a collection is indexed as its sequences joined by separators (code 0,
    // letters shifted up by one for the suffix array)
    std::vector<uint8_t> joined;
    const uint8_t *sa_codes = codes;
    int64_t J = n;
    int sa_sigma = ae_alphabet_sigma(alphabet);
    if (nseq > 0) {
        J = n + nseq - 1;
        try {
            joined.resize((size_t)J);
        } catch (...) {
            return AE_ENOMEM;
        }
        int64_t q = 0;
        for (int32_t k = 0; k < nseq; ++k) {
            const int64_t b = starts[k], e = k + 1 < nseq ? starts[k + 1] : n;
            if (k > 0) joined[q++] = 0;
            for (int64_t p = b; p < e; ++p) joined[q++] = (uint8_t)(codes[p] + 1);
        }
        sa_codes = joined.data();
        sa_sigma += 1;
    }
    const int64_t N = J + 1;
    std::vector<int32_t> sa;
    try {
        sa.resize((size_t)N);
    } catch (...) {
        return AE_ENOMEM;
    }
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return AE_ECUDA;
    }
    uint8_t *d_codes = nullptr;
    int32_t *d_sa = nullptr;
    ae_status res = AE_OK;
    if (cudaMalloc(&d_codes, (size_t)J) != cudaSuccess || cudaMalloc(&d_sa, sizeof(int32_t) * (size_t)N) != cudaSuccess) {
        cudaGetLastError();
        res = AE_ENOMEM;
    }
    if (res == AE_OK && cudaMemcpyAsync(d_codes, sa_codes, (size_t)J, cudaMemcpyHostToDevice, st) != cudaSuccess)
        res = AE_ECUDA;
    if (res == AE_OK) res = ae_sa_doubling(d_codes, J, sa_sigma, 1, d_sa, nullptr, st);
    if (res == AE_OK && (cudaMemcpyAsync(sa.data(), d_sa, sizeof(int32_t) * (size_t)N, cudaMemcpyDeviceToHost, st) !=
                             cudaSuccess ||
                         cudaStreamSynchronize(st) != cudaSuccess))
        res = AE_ECUDA;
    cudaStreamSynchronize(st);
    if (d_codes) cudaFree(d_codes);
    if (d_sa) cudaFree(d_sa);
    cudaStreamDestroy(st);
    if (res == AE_OK)
        res = nseq > 0 ? ae_host_index_fill_collection(codes, n, starts, nseq, alphabet, sa.data(), &idx->host)
                       : ae_host_index_fill(codes, n, alphabet, sa.data(), &idx->host);
    if (res == AE_OK) res = upload_index(idx);
    return res;
}

}  // namespace

extern "C" {

void ae_options_default(ae_options *opt) {
    if (!opt) return;
    opt->qprefix_seed = 1;
    opt->leaf_segment = 0;
    opt->item_columns = 1 << 24;
    opt->batch_columns = 1 << 20;
    opt->leaf_capacity = 4096;
    opt->profile = 0;
    opt->leaf_delay = 8;
    opt->int16_limit = 32000;
    opt->hint_hits = nullptr;
    opt->tier_stats = 0;
    opt->workspace_limit = 0;
    opt->general_rows = 0;
    opt->qprefix_domination = 1;
    opt->row_layout = 0;
    opt->fork_parts = 1;
    opt->leaf_wide_rows = 128;
    opt->fork_part = 0;
}

const char *ae_strerror(int32_t status) {
    switch (status) {
        case AE_OK: return "ok";
        case AE_EINVAL: return "invalid argument";
        case AE_ENOMEM: return "out of memory";
        case AE_EOVERFLOW: return "output buffer too small";
        case AE_ETIMEOUT: return "device wait timed out";
        case AE_ECUDA: return "CUDA runtime error";
        case AE_EUNSUPPORTED: return "unsupported size";
        case AE_EIO: return "index file error";
        default: return "unknown status";
    }
}

ae_status ae_suffix_array_device(const uint8_t *d_codes, int64_t n, int32_t sigma, int32_t reversed, int32_t *d_sa,
                                 void *stream) {
    if (n < 0 || sigma < 1 || sigma > 255 || (n > 0 && !d_codes) || !d_sa) return AE_EINVAL;
    if (n + 1 >= INT32_MAX) return AE_EUNSUPPORTED;
    return ae_sa_doubling(d_codes, n, sigma, reversed != 0, d_sa, nullptr, (cudaStream_t)stream);
}

ae_status ae_index_build(const uint8_t *text, int64_t n, int32_t alphabet, ae_index **out) {
    if (!out) return AE_EINVAL;
    *out = nullptr;
    if (!text || n < 1 || !ae_alphabet_sigma(alphabet)) return AE_EINVAL;
    if (n + 1 >= INT32_MAX) return AE_EUNSUPPORTED;
    std::vector<uint8_t> codes;
    try {
        codes.resize((size_t)n);
    } catch (...) {
        return AE_ENOMEM;
    }
    if (ae_encode_letters(text, n, alphabet, codes.data()) != 0) return AE_EINVAL;
    ae_index *idx = new (std::nothrow) ae_index();
    if (!idx) return AE_ENOMEM;
    ae_status st = build_index(idx, codes.data(), n, alphabet);
    if (st != AE_OK) {
        delete idx;
        return st;
    }
    *out = idx;
    return AE_OK;
}

ae_status ae_index_build_collection(const uint8_t *text, int64_t n, const int64_t *starts, int32_t nseq,
                                   int32_t alphabet, ae_index **out) {
    if (!out) return AE_EINVAL;
    *out = nullptr;
    if (!text || n < 1 || !starts || nseq < 1 || starts[0] != 0 || !ae_alphabet_sigma(alphabet)) return AE_EINVAL;
    for (int32_t k = 1; k < nseq; ++k)
        if (starts[k] < starts[k - 1] || starts[k] > n) return AE_EINVAL;
    if (n + nseq >= INT32_MAX) return AE_EUNSUPPORTED;
    std::vector<uint8_t> codes;
    try {
        codes.resize((size_t)n);
    } catch (...) {
        return AE_ENOMEM;
    }
    if (ae_encode_letters(text, n, alphabet, codes.data()) != 0) return AE_EINVAL;
    ae_index *idx = new (std::nothrow) ae_index();
    if (!idx) return AE_ENOMEM;
    ae_status st = build_index(idx, codes.data(), n, alphabet, starts, nseq);
    if (st != AE_OK) {
        delete idx;
        return st;
    }
    *out = idx;
    return AE_OK;
}

ae_status ae_index_save(const ae_index *idx, const char *path) {
    if (!idx || !path) return AE_EINVAL;
    return ae_host_index_save(&idx->host, path);
}

ae_status ae_index_load(const char *path, ae_index **out) {
    if (!path || !out) return AE_EINVAL;
    *out = nullptr;
    ae_index *idx = new (std::nothrow) ae_index();
    if (!idx) return AE_ENOMEM;
    ae_status st = ae_host_index_load(path, &idx->host);
    if (st == AE_OK) st = upload_index(idx);
    if (st != AE_OK) {
        delete idx;
        return st;
    }
    *out = idx;
    return AE_OK;
}

void ae_index_free(ae_index *idx) { delete idx; }

ae_status ae_index_info(const ae_index *idx, int64_t *n, int32_t *alphabet, int64_t *device_bytes) {
    if (!idx) return AE_EINVAL;
    if (n) *n = idx->host.n;
    if (alphabet) *alphabet = idx->host.alphabet;
    if (device_bytes) *device_bytes = idx->device_bytes;
    return AE_OK;
}

// The results of ae_search leave the device through pinned double buffers.  Up
// to OUT_THREADS host threads each copy a contiguous share of the hits in
// chunks of OUT_CHUNK bytes on their own stream, and move chunk k into the
// caller's buffer while chunk k + 1 is in flight.  A single copy into pageable
// memory goes through the CUDA runtime's own staging on one core and takes the fresh
// buffer's first-touch page faults one after another; here they are spread
// over the threads.  Small results take the single copy.
constexpr size_t OUT_CHUNK = (size_t)8 << 20;
constexpr int OUT_THREADS = 8;
constexpr size_t OUT_THREADED_MIN = (size_t)32 << 20;

static ae_status copy_hits_out(Workspace *w, ae_hit *h, const ae_hit *dev, int64_t total, cudaStream_t st) {
    const size_t bytes = sizeof(ae_hit) * (size_t)total;
    if (bytes < OUT_THREADED_MIN) {
        if (cudaMemcpyAsync(h, dev, bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return AE_ECUDA;
        return AE_OK;
    }
    int nt = (int)std::max(1u, std::min<unsigned>(OUT_THREADS, std::thread::hardware_concurrency()));
    nt = (int)std::min<size_t>((size_t)nt, (bytes + OUT_CHUNK - 1) / OUT_CHUNK);
    int dev_id = 0;
    if (cudaGetDevice(&dev_id) != cudaSuccess) return AE_ECUDA;
    const size_t need = (size_t)nt * 2 * OUT_CHUNK;
    if (w->h_out_bytes < need) {
        if (cudaStreamSynchronize(st) != cudaSuccess) return AE_ECUDA;
        if (w->h_out) cudaFreeHost(w->h_out);
        w->h_out = nullptr;
        w->h_out_bytes = 0;
        if (cudaMallocHost(&w->h_out, need) != cudaSuccess) return AE_ENOMEM;
        w->h_out_bytes = need;
    }
    while ((int)w->out_st.size() < nt) {
        // a thread's stream and its two events are kept only together
        cudaStream_t s = nullptr;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&e0, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&e1, cudaEventDisableTiming) != cudaSuccess) {
            if (e0) cudaEventDestroy(e0);
            if (s) cudaStreamDestroy(s);
            return AE_ECUDA;
        }
        w->out_st.push_back(s);
        w->out_ev.push_back(e0);
        w->out_ev.push_back(e1);
    }
    if (!w->out_ready && cudaEventCreateWithFlags(&w->out_ready, cudaEventDisableTiming) != cudaSuccess)
        return AE_ECUDA;
    if (cudaEventRecord(w->out_ready, st) != cudaSuccess) return AE_ECUDA;
    std::atomic<int> fail{0};
    auto share = [&](int t) {
        if (cudaSetDevice(dev_id) != cudaSuccess) {
            fail = 1;
            return;
        }
        cudaStream_t s = w->out_st[t];
        const size_t lo = sizeof(ae_hit) * ((size_t)total * t / nt);
        const size_t hi = sizeof(ae_hit) * ((size_t)total * (t + 1) / nt);
        const size_t nch = (hi - lo + OUT_CHUNK - 1) / OUT_CHUNK;
        uint8_t *buf[2] = {w->h_out + (size_t)(2 * t) * OUT_CHUNK, w->h_out + (size_t)(2 * t + 1) * OUT_CHUNK};
        auto issue = [&](size_t c) {
            const size_t o = lo + c * OUT_CHUNK, len = std::min(OUT_CHUNK, hi - o);
            return cudaMemcpyAsync(buf[c & 1], reinterpret_cast<const uint8_t *>(dev) + o, len,
                                   cudaMemcpyDeviceToHost, s) == cudaSuccess &&
                   cudaEventRecord(w->out_ev[2 * t + (c & 1)], s) == cudaSuccess;
        };
        bool ok = cudaStreamWaitEvent(s, w->out_ready, 0) == cudaSuccess && (nch == 0 || issue(0));
        for (size_t c = 0; ok && c < nch; ++c) {
            // chunk c + 1 goes into the buffer whose chunk c - 1 was moved out last round
            if (c + 1 < nch && !issue(c + 1)) ok = false;
            if (ok && cudaEventSynchronize(w->out_ev[2 * t + (c & 1)]) != cudaSuccess) ok = false;
            if (ok) {
                const size_t o = lo + c * OUT_CHUNK;
                memcpy(reinterpret_cast<uint8_t *>(h) + o, buf[c & 1], std::min(OUT_CHUNK, hi - o));
            }
        }
        // nothing may still be writing into the pinned chunks once this returns
        if (cudaStreamSynchronize(s) != cudaSuccess) ok = false;
        if (!ok) fail = 1;
    };
    std::vector<std::thread> th;
    th.reserve((size_t)nt);   // no reallocation (and no throw) once a thread runs
    int started = 1;
    try {
        for (; started < nt; ++started) th.emplace_back(share, started);
    } catch (const std::system_error &) {
        // no more threads: the shares not handed out are copied here
    }
    share(0);
    for (int t = started; t < nt; ++t) share(t);
    for (std::thread &x : th) x.join();
    return fail ? AE_ECUDA : AE_OK;
}

ae_status ae_search(const ae_index *idx, const ae_query *queries, int32_t nq, const ae_scoring *scoring,
                    const int32_t *H, const ae_options *opt, ae_hit **hits, int64_t *counts, void *stream) {
    if (!idx || !hits || !counts || nq < 0 || (nq > 0 && (!queries || !H))) return AE_EINVAL;
    *hits = nullptr;
    if (nq == 0) return AE_OK;
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<int64_t> off(nq + 1, 0);
    for (int q = 0; q < nq; ++q) {
        if (queries[q].len < 0 || (queries[q].len > 0 && !queries[q].seq)) return AE_EINVAL;
        off[q + 1] = off[q] + queries[q].len;
    }
    try {
        Workspace *w = workspace_for(idx, st);
        std::lock_guard<std::mutex> busy(w->busy);
        const int64_t total_len = off[nq];
        uint8_t *h_ascii = nullptr;
        if (total_len > 0) {
            if ((size_t)total_len > w->h_stage_bytes) {
                CU(cudaStreamSynchronize(st));
                if (w->h_stage) cudaFreeHost(w->h_stage);
                w->h_stage = nullptr;
                w->h_stage_bytes = 0;
                size_t nb = std::max((size_t)total_len, w->h_stage_bytes + w->h_stage_bytes / 4);
                nb = std::max<size_t>(nb, 1 << 16);
                CU(cudaMallocHost(&w->h_stage, nb));
                w->h_stage_bytes = nb;
            }
            h_ascii = w->h_stage;
            for (int q = 0; q < nq; ++q)
                if (queries[q].len) memcpy(h_ascii + off[q], queries[q].seq, (size_t)queries[q].len);
        }
        ensure(w->ascii, std::max<int64_t>(total_len, 1), st);
        ensure(w->codes, std::max<int64_t>(total_len, 1), st);
        ensure(w->bad, 4, st);
        CU(cudaMemsetAsync(w->bad.p, 0, 4, st));
        if (total_len > 0)
            CU(cudaMemcpyAsync(w->ascii.p, h_ascii, (size_t)total_len, cudaMemcpyHostToDevice, st));
        ae_encode_queries(ptr<uint8_t>(w->ascii), ptr<uint8_t>(w->codes), total_len, idx->host.alphabet,
                          ptr<int>(w->bad), st);
        int bad = 0;
        CU(cudaMemcpyAsync(&bad, w->bad.p, 4, cudaMemcpyDeviceToHost, st));
        CU(cudaStreamSynchronize(st));
        if (bad) return AE_EINVAL;
        ae_hit *dev = nullptr;
        std::vector<int64_t> cnt;
        int64_t total = 0;
        ae_status e = search_core(idx, w, off.data(), nq, scoring, H, opt, st, &dev, cnt, &total);
        if (e != AE_OK) return e;
        ae_hit *h = (ae_hit *)malloc(sizeof(ae_hit) * (size_t)std::max<int64_t>(total, 1));
        if (!h) return AE_ENOMEM;
        if (total > 0) {
            const ae_status ce = copy_hits_out(w, h, dev, total, st);
            if (ce != AE_OK) {
                free(h);
                return ce;
            }
        }
        for (int q = 0; q < nq; ++q) counts[q] = cnt[q];
        *hits = h;
    } catch (const ae_error &err) {
        cudaGetLastError();
        return err.st;
    } catch (const std::bad_alloc &) {
        return AE_ENOMEM;
    }
    return AE_OK;
}

void ae_hits_free(ae_hit *hits) { free(hits); }

ae_status ae_search_device(const ae_index *idx, const uint8_t *d_seq, const int64_t *offsets, int32_t nq,
                           const ae_scoring *scoring, const int32_t *H, const ae_options *opt, ae_hit *d_hits,
                           int64_t capacity, int64_t *counts, void *stream) {
    if (!idx || !offsets || !counts || nq < 0 || (nq > 0 && !H) || capacity < 0 || (capacity > 0 && !d_hits))
        return AE_EINVAL;
    if (nq == 0) return AE_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t total_len = offsets[nq] - offsets[0];
    if (offsets[0] != 0 || total_len < 0) return AE_EINVAL;
    try {
        Workspace *w = workspace_for(idx, st);
        std::lock_guard<std::mutex> busy(w->busy);
        ensure(w->codes, std::max<int64_t>(total_len, 1), st);
        ensure(w->bad, 4, st);
        CU(cudaMemsetAsync(w->bad.p, 0, 4, st));
        if (total_len > 0 && !d_seq) return AE_EINVAL;
        ae_encode_queries(d_seq, ptr<uint8_t>(w->codes), total_len, idx->host.alphabet, ptr<int>(w->bad), st);
        int bad = 0;
        CU(cudaMemcpyAsync(&bad, w->bad.p, 4, cudaMemcpyDeviceToHost, st));
        CU(cudaStreamSynchronize(st));
        if (bad) return AE_EINVAL;
        ae_hit *dev = nullptr;
        std::vector<int64_t> cnt;
        int64_t total = 0;
        ae_status e = search_core(idx, w, offsets, nq, scoring, H, opt, st, &dev, cnt, &total);
        if (e != AE_OK) return e;
        for (int q = 0; q < nq; ++q) counts[q] = cnt[q];
        if (total > capacity) return AE_EOVERFLOW;
        if (total > 0) {
            CU(cudaMemcpyAsync(d_hits, dev, sizeof(ae_hit) * (size_t)total, cudaMemcpyDeviceToDevice, st));
            CU(cudaStreamSynchronize(st));
        }
    } catch (const ae_error &err) {
        cudaGetLastError();
        return err.st;
    } catch (const std::bad_alloc &) {
        return AE_ENOMEM;
    }
    return AE_OK;
}

ae_status ae_hits_merge(const ae_hit *d_hits, const int32_t *d_qid, int64_t n, int32_t nq, int64_t text_len,
                        int64_t max_query_len, ae_hit *d_out, int64_t *counts, int64_t *total, void *stream) {
    if (n < 0 || nq < 1 || text_len < 1 || max_query_len < 1 || !counts || !total || (n > 0 && (!d_hits || !d_qid || !d_out)))
        return AE_EINVAL;
    const int be = bits_for(std::max<int64_t>(text_len - 1, 1)), bj = bits_for(std::max<int64_t>(max_query_len - 1, 1));
    const int bq = bits_for(std::max(nq - 1, 1));
    if (be + bj + bq > 64) return AE_EUNSUPPORTED;
    for (int32_t q = 0; q < nq; ++q) counts[q] = 0;
    *total = 0;
    if (n == 0) return AE_OK;
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<void *> bufs;
    auto alloc = [&](size_t bytes) -> void * {
        void *p = nullptr;
        if (cudaMalloc(&p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
            cudaGetLastError();
            throw ae_error{AE_ENOMEM};
        }
        bufs.push_back(p);
        return p;
    };
    ae_status res = AE_OK;
    try {
        uint64_t *k0 = (uint64_t *)alloc(8 * (size_t)n), *k1 = (uint64_t *)alloc(8 * (size_t)n);
        uint32_t *v0 = (uint32_t *)alloc(4 * (size_t)n), *v1 = (uint32_t *)alloc(4 * (size_t)n);
        uint64_t *tmp = (uint64_t *)alloc(8 * (size_t)std::max(ae_sort_tmp_words(n), ae_scan_tmp_words(n, 1)));
        uint32_t *flags = (uint32_t *)alloc(4 * (size_t)n);
        uint64_t *off = (uint64_t *)alloc(8 * (size_t)n), *tot = (uint64_t *)alloc(64);
        unsigned long long *qc = (unsigned long long *)alloc(8 * (size_t)nq);
        CU(cudaMemsetAsync(qc, 0, 8 * (size_t)nq, st));
        ae_merge_keys(d_hits, d_qid, n, be, bj, k0, v0, st);
        const int which = ae_radix_sort(k0, v0, k1, v1, n, be + bj + bq, tmp, st);
        const uint64_t *keys = which ? k1 : k0;
        const int32_t *scores = (const int32_t *)(which ? v1 : v0);
        ae_unique_flags(keys, n, flags, st);
        const uint32_t *in[1] = {flags};
        uint64_t *out[1] = {off};
        ae_scan_u32(in, out, 1, n, tot, tmp, st);
        ae_unique_write(keys, scores, n, off, be, bj, d_out, qc, st);
        std::vector<unsigned long long> hq(nq);
        uint64_t u = 0;
        CU(cudaMemcpyAsync(&u, tot, 8, cudaMemcpyDeviceToHost, st));
        CU(cudaMemcpyAsync(hq.data(), qc, 8 * (size_t)nq, cudaMemcpyDeviceToHost, st));
        CU(cudaStreamSynchronize(st));
        CU(cudaGetLastError());
        for (int32_t q = 0; q < nq; ++q) counts[q] = (int64_t)hq[q];
        *total = (int64_t)u;
    } catch (const ae_error &e) {
        cudaStreamSynchronize(st);
        cudaGetLastError();
        res = e.st;
    }
    for (void *p : bufs) cudaFree(p);
    return res;
}

ae_status ae_workspace_info(const ae_index *idx, void *stream, int64_t *bytes, int64_t *process_bytes) {
    if (!idx) return AE_EINVAL;
    ae_index *x = const_cast<ae_index *>(idx);
    int64_t b = 0;
    {
        std::lock_guard<std::mutex> g(x->mu);
        for (auto &p : x->ws)
            if (p.first == (cudaStream_t)stream) {
                std::lock_guard<std::mutex> busy(p.second->busy);
                b = p.second->device_bytes();
            }
    }
    if (bytes) *bytes = b;
    if (process_bytes) *process_bytes = g_ws_bytes.load();
    return AE_OK;
}

ae_status ae_workspace_release(ae_index *idx, void *stream) {
    if (!idx) return AE_EINVAL;
    Workspace *w = nullptr;
    {
        std::lock_guard<std::mutex> g(idx->mu);
        for (size_t k = 0; k < idx->ws.size(); ++k)
            if (idx->ws[k].first == (cudaStream_t)stream) {
                w = idx->ws[k].second;
                idx->ws.erase(idx->ws.begin() + (long)k);
                break;
            }
    }
    if (!w) return AE_OK;
    {
        // wait for a search still running on this stream in another thread
        std::lock_guard<std::mutex> busy(w->busy);
        if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) {
            cudaGetLastError();
        }
    }
    delete w;
    return AE_OK;
}

ae_status ae_last_stats(ae_stats *out) {
    if (!out) return AE_EINVAL;
    *out = g_last_stats;
    return AE_OK;
}

ae_status ae_plan(int64_t m, int32_t alphabet, const ae_scoring *scoring, int32_t H, int32_t *q,
                  int32_t *seed_depth_out, int64_t *L_max) {
    const int sigma = ae_alphabet_sigma(alphabet);
    if (!scoring || m < 0 || H < 1 || !sigma) return AE_EINVAL;
    ScoreView sc;
    ae_status e = make_score(scoring, sigma, sc);
    if (e != AE_OK) return e;
    if (q) *q = sc.use_matrix ? 0 : std::min(-sc.sb, -(sc.sg + sc.ss)) / sc.sa + 1;
    if (seed_depth_out) *seed_depth_out = seed_depth(sc, H, true);
    if (L_max) {
        // Eq. 1: L_max = max{m, m + floor((H - (s_a m + s_g)) / s_s)}, mathematical floor
        int64_t num = (int64_t)H - ((int64_t)sc.sa * m + sc.sg);
        int64_t den = sc.ss;  // < 0
        int64_t qv = num / den;
        if ((num % den != 0) && ((num < 0) != (den < 0))) --qv;
        *L_max = std::max<int64_t>(m, m + qv);
    }
    return AE_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ no-allocation search
//
// ae_search_device_static: the search of ae_search_device for callers that
// must not allocate device memory (e.g. a host process whose device memory is
// fully reserved by another allocator).  Every working buffer of the
// search -- level arenas, sort buffers, hit records and the per-warp rows of
// the text-position sweep -- is carved from one file-scope device array of
// AE_STATIC_SCRATCH_BYTES, which every GPU that loads this library holds
// until the process exits.

namespace {

constexpr size_t AE_STATIC_SCRATCH_BYTES = (size_t)64 << 20;
constexpr int64_t AE_STATIC_MAX_COLUMNS = 65536;
constexpr int32_t AE_STATIC_MAX_QUERIES = 4096;
constexpr int AE_STATIC_MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_ae_static_scratch[AE_STATIC_SCRATCH_BYTES];

// Host-side state per device: the device address of the array (the array's
// name in host code is only a stand-in for the symbol), the workspace whose
// buffers point into it, and a host staging area.
void *g_static_ptr[AE_STATIC_MAX_DEVICES];
Workspace g_static_ws[AE_STATIC_MAX_DEVICES];
uint64_t g_static_htot[AE_STATIC_MAX_DEVICES][64];
std::mutex g_static_mu[AE_STATIC_MAX_DEVICES];

// Grow buffer b to at least `bytes` inside the arena, keeping its first `keep`
// bytes.  The most recently carved buffer grows in place; any other buffer gets
// a new region 1.25x larger than it was (as ensure() grows), so a buffer that
// grows level by level in small steps does not use up the array early.
void carve(DevBuf &b, size_t bytes, size_t keep, cudaStream_t st) {
    StaticArena &a = *g_arena;
    if (b.carved && b.p && reinterpret_cast<char *>(b.p) + b.bytes == a.base + a.used) {
        const size_t start = (size_t)(reinterpret_cast<char *>(b.p) - a.base);
        if (start + bytes > a.cap) throw ae_error{AE_EUNSUPPORTED};
        a.used = start + bytes;
        b.bytes = bytes;
        return;
    }
    const size_t off = (a.used + 255) & ~size_t(255);
    size_t nb = std::max(bytes, b.bytes + b.bytes / 4);
    if (off + nb > a.cap) nb = bytes;   // the growth margin is optional, the request is not
    if (off + nb > a.cap) throw ae_error{AE_EUNSUPPORTED};
    void *p = a.base + off;
    if (keep && b.p) CU(cudaMemcpyAsync(p, b.p, keep, cudaMemcpyDeviceToDevice, st));
    a.used = off + nb;
    b.p = p;
    b.bytes = nb;
    b.carved = true;
}

}  // namespace

extern "C" ae_status ae_search_device_static(const ae_index *idx, const uint8_t *d_seq, const int64_t *offsets,
                                             int32_t nq, const ae_scoring *scoring, const int32_t *H,
                                             const ae_options *opt, ae_hit *d_hits, int64_t capacity,
                                             int64_t *counts, void *stream) {
    if (!idx || !offsets || !counts || nq < 0 || (nq > 0 && !H) || capacity < 0 || (capacity > 0 && !d_hits))
        return AE_EINVAL;
    if (nq == 0) return AE_OK;
    const int64_t total_len = offsets[nq] - offsets[0];
    if (offsets[0] != 0 || total_len < 0) return AE_EINVAL;
    if (total_len > 0 && !d_seq) return AE_EINVAL;
    if (total_len > AE_STATIC_MAX_COLUMNS || nq > AE_STATIC_MAX_QUERIES) return AE_EUNSUPPORTED;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return AE_ECUDA;
    }
    if (dev < 0 || dev >= AE_STATIC_MAX_DEVICES) return AE_EUNSUPPORTED;
    cudaStream_t st = (cudaStream_t)stream;
    std::lock_guard<std::mutex> guard(g_static_mu[dev]);
    if (!g_static_ptr[dev]) {
        // once per device, with that device current
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_ae_static_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return AE_ECUDA;
        }
        g_static_ptr[dev] = p;
    }
    ae_options o;
    ae_options_default(&o);
    if (opt) o = *opt;
    o.profile = 0;
    o.leaf_capacity = std::max(64, std::min(o.leaf_capacity, 256));
    Workspace &w = g_static_ws[dev];
    w.forget_carved();
    w.stream = st;
    w.h_tot = g_static_htot[dev];
    w.h_tot_static = true;
    w.leaf_cap = 0;
    StaticArena arena{reinterpret_cast<char *>(g_static_ptr[dev]), AE_STATIC_SCRATCH_BYTES, 0};
    g_arena = &arena;
    ae_status status = AE_OK;
    try {
        ensure(w.codes, std::max<int64_t>(total_len, 1), st);
        ensure(w.bad, 4, st);
        CU(cudaMemsetAsync(w.bad.p, 0, 4, st));
        ae_encode_queries(d_seq, ptr<uint8_t>(w.codes), total_len, idx->host.alphabet, ptr<int>(w.bad), st);
        CU(cudaMemcpyAsync(w.h_tot, w.bad.p, 4, cudaMemcpyDeviceToHost, st));
        CU(cudaStreamSynchronize(st));
        if (*reinterpret_cast<int *>(w.h_tot)) {
            status = AE_EINVAL;
        } else {
            ae_hit *dev_hits = nullptr;
            std::vector<int64_t> cnt;
            int64_t total = 0;
            status = search_core(idx, &w, offsets, nq, scoring, H, &o, st, &dev_hits, cnt, &total);
            if (status == AE_OK) {
                for (int q = 0; q < nq; ++q) counts[q] = cnt[q];
                if (total > capacity) {
                    status = AE_EOVERFLOW;
                } else if (total > 0) {
                    CU(cudaMemcpyAsync(d_hits, dev_hits, sizeof(ae_hit) * (size_t)total, cudaMemcpyDeviceToDevice,
                                       st));
                    CU(cudaStreamSynchronize(st));
                }
            }
        }
    } catch (const ae_error &err) {
        status = err.st;
    } catch (const std::bad_alloc &) {
        status = AE_ENOMEM;
    }
    // A search that stopped early (the array ran out, a CUDA call failed) may
    // still have kernels queued that write into the array: wait for them while
    // the device's lock is held, so the next call never shares the array with them.
    cudaStreamSynchronize(st);
    cudaGetLastError();
    g_arena = nullptr;
    return status;
}
