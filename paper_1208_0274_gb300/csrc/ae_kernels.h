// Launch wrappers of the device kernels (ae_kernels.cu), called by the engine.
#pragma once

#include <cuda_runtime.h>

#include "ae_internal.h"

// Number of kernel launches issued so far by the calling thread.
int64_t ae_launches_read();
extern thread_local int64_t g_launches;

// Exclusive scans of W u32 arrays of length N into u64 arrays; totals[w]
// (device, W entries) receives the sums.  tmp must hold scan_tmp_words(N, W)
// u64 words.
int64_t ae_scan_tmp_words(int64_t N, int W);
void ae_scan_u32(const uint32_t *const *in, uint64_t *const *out, int W, int64_t N, uint64_t *totals,
                 uint64_t *tmp, cudaStream_t st);

// Stable LSD radix sort of (key, value) pairs on the low `bits` bits of the
// key.  Ping-pong buffers k0/v0 (input) and k1/v1; returns 0 if the result
// ended in k0/v0, 1 if in k1/v1.  tmp must hold ae_sort_tmp_words(N) u64.
int64_t ae_sort_tmp_words(int64_t N);
int ae_radix_sort(uint64_t *k0, uint32_t *v0, uint64_t *k1, uint32_t *v1, int64_t N, int bits,
                  uint64_t *tmp, cudaStream_t st);

// Suffix array of the n codes at d_codes (read backwards with `reversed`)
// followed by a unique smallest sentinel, into d_sa[0..n] (device), by prefix
// doubling; *rounds receives the number of radix sorts.  Allocates and frees
// its work buffers; returns after `st` has finished.  AE_EINVAL on a code >=
// sigma, AE_ENOMEM, AE_ECUDA.
ae_status ae_sa_doubling(const uint8_t *d_codes, int64_t n, int sigma, int reversed, int32_t *d_sa, int *rounds,
                         cudaStream_t st);

// Query letters -> codes; sets *bad (device int) on an unknown letter.
void ae_encode_queries(const uint8_t *ascii, uint8_t *codes, int64_t total, int alphabet, int *bad,
                       cudaStream_t st);

struct SeedArgs {
    IndexView ix;
    ScoreView sc;
    QueryView qv;
    const WorkItem *items;
    const int64_t *item_pos;   // exclusive prefix of seed positions per item (nitems + 1)
    int32_t nitems;
    int32_t d0;                // seed depth (>= 1)
    int64_t npos;
    int32_t int16;             // 1: write the seed rows as packed int16x2 pairs into aM
    // q-prefix domination (Lemma 1): per d0-gram (packed as in the seed keys) the
    // mask of letters that precede its occurrences in T (bit sigma: an occurrence
    // starting a sequence); NULL = off.  `dominated` counts the dropped entries.
    const uint32_t *dom;
    unsigned long long *dominated;
    // fork partition (one query's search split over ranks): with parts > 1 only
    // the seed grams whose hash falls in part `part` start forks here
    int32_t parts, part;
};
// Predecessor masks of every d0-gram of the text (the table SeedArgs::dom reads):
// mask[gram] |= 1 << (letter before the occurrence, or sigma at a sequence start).
// mask must hold sigma_bits^d0 words and be zeroed.
void ae_dom_table(const IndexView &ix, int d0, uint32_t *mask, cudaStream_t st);
// keys = (item << 2*d0... packed gram), vals = query start column y.
void ae_seed_keys(const SeedArgs &a, uint64_t *keys, uint32_t *vals, cudaStream_t st);
// After sorting: one node per run of equal keys; writes nodes + level-0 arena.
// Returns via *nnodes (device u64).
void ae_seed_nodes(const SeedArgs &a, const uint64_t *keys, const uint32_t *vals, int64_t npos, int key_bits,
                   uint32_t *flags, uint64_t *flag_off, uint64_t *tmp, Node *nodes, int32_t *aj, int32_t *aM,
                   int32_t *aGa, uint64_t *nnodes_dev, cudaStream_t st);

// ---- one trie level (ae_trie.cu)
struct ChildrenArgs {
    IndexView ix;
    const WorkItem *items;
    const Node *nodes;
    int64_t nnodes;
    uint32_t *nseg, *ntrip;               // per node: non-empty children, triples
    DevStats *stats;
};
void ae_children(const ChildrenArgs &a, cudaStream_t st);

// A non-empty child (32 bytes): SA range, row length (= parent entries; bits
// 0-27 of len, bits 28-31 = levels the parent has been a single occurrence),
// first triple, and either the parent row's offset or, for the implicit root
// row, the work item's columns [c0, c1) packed as c0 | c1 << 32.  cq packs the
// letter (bits 0-4), the query id (bits 5-28) and the root flag (bit 31).
struct Seg {
    uint32_t lo, hi;
    uint32_t len, cq;
    uint64_t toff;
    uint64_t poff;
};
// Triples per k_rows task window.  A task takes the segments that start in
// its window (the last one may run past it).
// (192: the largest window whose per-warp tables leave room for 6 resident
// blocks of 8 warps; measured best on the 100 Mbp workload)
#ifndef AE_ROW_TASK_TRIPLES
#define AE_ROW_TASK_TRIPLES 192
#endif
constexpr int AE_ROW_TASK = AE_ROW_TASK_TRIPLES;
// k_compact also writes task_first[w] = the first segment starting at or
// after triple w * AE_ROW_TASK, for every window w < ceil(triples / AE_ROW_TASK).
void ae_compact_segs(const ChildrenArgs &a, const uint64_t *seg_off, const uint64_t *trip_off, Seg *segs,
                     uint64_t *task_first,
                     cudaStream_t st);

// Counters of one level: totals from the count pass (c_*), reservation
// cursors of the write pass, and the two passes' task counters.
struct LevelCounters {
    unsigned long long c_fr_ent, c_fr_node, c_lf_ent, c_lf_node, c_hits;
    unsigned long long fr_ent, fr_node, lf_ent, lf_node, hits;
    unsigned long long overflow, task_c, task_w, wide;   // wide: a task total passed 2^32 - 1
    unsigned long long triples;   // DNA int16x2 route: (child, parent entry) pairs of the level
    unsigned long long retry;     // DNA int16x2 route: a reservation passed an arena's capacity
};

struct RowsArgs {
    IndexView ix;
    ScoreView sc;
    QueryView qv;
    const WorkItem *items;
    const Node *nodes;
    const int32_t *pj, *pM, *pGa;         // parent arena
    const Seg *segs;
    const uint64_t *nseg_dev, *ntrip_dev; // scan totals (device)
    int32_t *fj, *fM, *fGa;               // next-level arena
    Node *fnodes;
    uint64_t fr_ent_cap, fr_node_cap;
    int32_t *lj, *lM, *lGa;               // leaf arena (accumulates over levels)
    Inject *inj;
    uint64_t lf_ent_cap, lf_node_cap;
    RangeHit *rhits;
    uint64_t hit_cap;
    LevelCounters *ctr;
    DevStats *stats;
    int32_t leaf_delay;                   // levels a single-occurrence child stays in the walk
    uint32_t *seg_cnt, *seg_hit;          // per segment: outputs and hits (count pass -> write pass)
    const uint64_t *task_first;           // per task window: its first segment (from k_compact)
    // count pass: per task and arena kind (fr_ent, lf_ent, fr_node, lf_node, hits) its output
    // count, at task_tot[kind * task_stride + task]; write pass: their exclusive scan task_off
    // (or NULL: reserve with atomics on ctr) plus the level bases base_off[kind]
    uint32_t *task_tot;
    const uint64_t *task_off;
    uint64_t task_stride;
    uint64_t base_off[5];
    int32_t int16;                        // 1: parent and frontier rows are packed int16x2 (M | G_a << 16) in pM / fM
    int32_t tiers;                        // 1: count entries by cost tier (ae_stats.entries_tier)
    int32_t parts, part;                  // root rows: with parts > 1 only start columns j with
                                          // j % parts == part open forks (a search split over ranks)
    // int16x2 route without tier counting: per triple the final slot values of the count
    // pass (M_A | M_B << 16, 0 = dead) and the key K of its gap run (AE_KNEG: none)
    uint32_t *res;
    int32_t *res_key;
};
void ae_rows(const RowsArgs &a, bool write, int blocks, cudaStream_t st);
int ae_rows_blocks_per_sm(bool write);   // blocks per SM to launch a k_rows pass with (one full wave)
void ae_mg_to_i32(int32_t *M, int32_t *Ga, int64_t n, cudaStream_t st);

// ---- one trie level of the DNA int16x2 route in one launch (ae_rows_dna.cu).
// Tasks are groups of nodes_per_task (<= 32) nodes whose child ranges are
// taken in the task's prologue; each task counts its outputs, reserves its
// ranges on the level cursors of `ctr` (fr_ent, lf_ent, fr_node, lf_node,
// hits, uploaded at the arenas' bases) and writes them.  A reservation past a
// capacity raises ctr->retry and leaves the task unwritten; the cursors end at
// the level's exact totals either way.  The output arguments are those of
// RowsArgs.
struct DnaRowsArgs {
    IndexView ix;
    ScoreView sc;
    QueryView qv;
    const Node *nodes;
    int64_t nnodes;
    int32_t nodes_per_task;
    int32_t leaf_delay;
    uint64_t urec;                        // ceil(2^32 / u), u = -s_s: gap-run lengths without division
    int32_t sequential;                   // 1: one lane per (node, child) walking the parent row in order
                                          // (short rows); 0: one lane per parent entry (long rows)
    const int32_t *pj;                    // parent arena: column, packed (M | G_a << 16)
    const uint32_t *pmg;
    int32_t *fj;                          // next-level arena (packed rows)
    uint32_t *fmg;
    Node *fnodes;
    uint64_t fr_ent_cap, fr_node_cap;
    int32_t *lj, *lM, *lGa;               // leaf arena (int32 rows)
    Inject *inj;
    uint64_t lf_ent_cap, lf_node_cap;     // absolute: the leaf arenas accumulate over levels
    RangeHit *rhits;
    uint64_t hit_cap;
    LevelCounters *ctr;
    // walk layout: the count phase keeps each pair's child row here (per warp and
    // lane, stage_cap entries of (column, packed M | G_a)); rows that fit are
    // copied out after the reservation instead of being computed again.  NULL:
    // every row is computed twice
    uint2 *stage;
    int32_t stage_cap;
};
void ae_rows_dna(const DnaRowsArgs &a, int blocks, cudaStream_t st);
int ae_rows_dna_blocks_per_sm();
int ae_rows_dna_warps_per_block();
struct LeafArgs {
    IndexView ix;
    ScoreView sc;
    QueryView qv;
    const Inject *inj;
    const uint32_t *order;        // injections sorted by (qid, e)
    int64_t ninj;
    const int32_t *lj, *lM, *lGa; // leaf arena
    int32_t seg;
    int64_t nseg;
    unsigned long long *next_seg;
    int32_t *scratch;
    int32_t cap;
    int32_t nwarps;
    uint64_t *hit_key;
    int32_t *hit_score;
    unsigned long long *hit_count;
    uint64_t hit_cap;
    int32_t be, bj;               // key packing widths
    int32_t tiers;                // 1: count entries by cost tier
    DevStats *stats;
    // walks whose row grows past esc_min entries (0: never) continue on a whole
    // block (k_leaf_wide) with the rest of their task's injections, in one of
    // esc_max slots: esc[slot] the walk's state, esc_rows + slot * 12 * cap its
    // four row buffers; *esc_count counts the slots taken (it may pass esc_max:
    // a walk that finds no free slot stays on its warp)
    int32_t esc_min, esc_max;
    unsigned long long *esc_count;
    struct EscWalk *esc;
    int32_t *esc_rows;
};
// A sweep walk handed from a warp to a block: its query, text position, the
// row at that position (in the slot's first buffer) and its task's remaining
// injections [k, kend) (indices into the sorted order).
struct EscWalk {
    int32_t qid, p;
    int64_t rlen, k, kend;
};
void ae_inject_keys(const Inject *inj, int64_t ninj, uint64_t *keys, uint32_t *vals, cudaStream_t st);
void ae_leaf_sweep(const LeafArgs &a, int blocks, int threads, cudaStream_t st);
int64_t ae_leaf_scratch_words(int32_t cap, int32_t nwarps);

// Range hits -> point hits (key, score) appended at dst.
void ae_locate_counts(const RangeHit *rh, int64_t nrh, uint32_t *cnt, cudaStream_t st);
void ae_locate(const RangeHit *rh, int64_t nrh, const uint64_t *off, int64_t total, const int32_t *tend, int be,
               int bj, uint64_t *key, int32_t *score, cudaStream_t st);

// Result records (with per-record query ids) -> sort keys (query, text end, query end) and scores.
void ae_merge_keys(const ae_hit *hits, const int32_t *qid, int64_t N, int be, int bj, uint64_t *key, uint32_t *val,
                   cudaStream_t st);

// Sorted (key, score) -> unique keys with max score.
void ae_unique_flags(const uint64_t *key, int64_t N, uint32_t *flags, cudaStream_t st);
void ae_unique_compact(const uint64_t *key, const int32_t *score, int64_t N, const uint64_t *flag_off, uint64_t *okey,
                       int32_t *oscore, cudaStream_t st);
void ae_unique_write(const uint64_t *key, const int32_t *score, int64_t N, const uint64_t *flag_off, int be,
                     int bj, ae_hit *out, unsigned long long *qcount, cudaStream_t st);
