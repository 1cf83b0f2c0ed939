/*
 * ae.h — C ABI of the GB300 exact local-alignment search library (libae.so).
 *
 * The library answers the local-alignment problem of Section 2.1: for a text T
 * (n letters) and a query P (m letters), every pair (text end i, query end j)
 * whose largest similarity max_{x<=i, y<=j} sim(T[x..i], P[y..j]) reaches a
 * threshold H, with sim the best global-alignment score under an affine-gap
 * scheme (Algorithm 1's output A(i,j) >= H).  It walks the suffix trie of T
 * through an FM index of the reversed text (Section 5), computes one Gotoh row
 * per trie node (Section 2.2) and skips the entries that Theorems 1-3 prove
 * meaningless (Section 3.1).
 *
 * Conventions
 *  - Letters are ASCII: DNA "ACGT" (upper case), protein the 20 residues
 *    "ARNDCQEGHILKMFPSTWYV".  Any other byte is an error (AE_EINVAL).
 *  - Positions are 0-based, ends inclusive (the paper is 1-based: pi = end+1).
 *  - Every entry point returns an ae_status; no C++ exception crosses the ABI.
 *  - Host pointers are marked "host", device pointers "device" (CUDA global
 *    memory of the current device).  The library never frees caller memory.
 *  - An ae_index is immutable after build/load and may be shared by threads;
 *    run at most one search per stream at a time.
 */
#ifndef AE_H
#define AE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    AE_OK = 0,
    AE_EINVAL = 1,        /* bad argument: scheme signs, H < 1, unknown letter, empty text */
    AE_ENOMEM = 2,        /* host or device allocation failed */
    AE_EOVERFLOW = 3,     /* caller buffer too small; required sizes are returned */
    AE_ETIMEOUT = 4,      /* a bounded device wait gave up */
    AE_ECUDA = 5,         /* a CUDA runtime call failed */
    AE_EUNSUPPORTED = 6,  /* sizes beyond the library's limits (e.g. n >= 2^31) */
    AE_EIO = 7            /* file read/write or format error */
} ae_status;

enum { AE_DNA = 0, AE_PROTEIN = 1 };

typedef struct ae_index ae_index;   /* opaque; owns its device memory */

/* Scoring scheme <s_a, s_b, s_g, s_s> of Section 2.1: an identical pair scores
 * match (> 0), a substitution mismatch (< 0), a run of r gap letters scores
 * gap_open + r * gap_extend (gap_open <= 0, gap_extend < 0).  If matrix is not
 * NULL it is a host sigma x sigma table (row = text letter, column = query
 * letter, alphabet order above) used instead of match/mismatch; its diagonal
 * must be positive.  With a matrix the q-prefix seeding of Theorem 3 is off
 * and the trie walk starts at the root. */
typedef struct {
    int32_t match;
    int32_t mismatch;
    const int8_t *matrix;
    int32_t gap_open;
    int32_t gap_extend;
} ae_scoring;

/* One result: the largest similarity `score` of any alignment ending at text
 * position text_end and query position query_end (a result of Algorithm 1). */
typedef struct {
    int64_t text_end;
    int32_t query_end;
    int32_t score;
} ae_hit;

typedef struct {
    const uint8_t *seq;   /* host ASCII letters */
    int64_t len;
} ae_query;

/* Counters of the last search on the calling thread, summed over queries.
 * The tiers follow Table 4's cost model: an entry whose value came from one
 * live term of the recurrence (the no-gap form of Eq. 3) costs 1, from two
 * live terms 2, from all three 3. */
typedef struct {
    int64_t nodes;          /* trie nodes whose rows were computed (range size >= 2) */
    int64_t leaf_rows;      /* rows computed along unique text positions */
    int64_t entries;        /* live DP entries written */
    int64_t entries_tier[3];   /* with ae_options.tier_stats: trie entries by cost tier */
    int64_t injections;     /* trie rows handed to the text-position sweep */
    int64_t raw_hits;       /* hit records before the per-cell max */
    int64_t hits;           /* distinct (query, text end, query end) results */
    int64_t entries_leaf;   /* of `entries`, those written by the text-position sweep */
    int64_t launches;       /* kernel launches issued by the search */
    int32_t levels;         /* trie levels expanded */
    int32_t levels_int16;   /* of them, levels whose rows were int16x2 pairs */
    int32_t seed_depth;     /* depth the trie walk started at */
    double  ms_trie, ms_leaf, ms_reduce, ms_total;   /* host wall time per phase */
    /* with ae_options.profile: device time of the kernels, by kind, from CUDA
     * events recorded on the search's stream around each launch group:
     * ms_k_rows = the row kernel of the trie levels, ms_k_expand = the child
     * ranges with their scan and compaction, ms_k_leaf = the text-position
     * sweep, ms_k_sort = radix sorts, ms_k_other = the rest */
    double  ms_k_expand, ms_k_leaf, ms_k_sort, ms_k_other, ms_k_rows;
    int64_t leaf_max_steps;   /* longest text walk of one sweep task (positions) */
    int64_t leaf_max_width;   /* widest row met by the sweep (entries) */
    int64_t ws_bytes;         /* device bytes held by the library's working buffers */
    int64_t leaf_sweeps;      /* launches of the text-position sweep (one per batch, plus one per
                                 rerun after its hit buffer or a row buffer overflowed) */
    int64_t leaf_raw_hits;    /* hit records written by the sweep (before the per-cell max) */
    int64_t triples;          /* (child, parent entry) pairs the trie levels evaluated: every
                                 non-empty child of a node with every entry of the node's row */
    int64_t batch_splits;     /* batches that ran out of device memory and were searched again
                                 as two halves (the result is the same) */
    int64_t dominated;        /* forks dropped at the seed depth by q-prefix domination (Lemma 1):
                                 the text letter before every occurrence of the seed gram equals
                                 the query letter before the fork's start */
    /* Filtering and reuse (Section 7.2, Eq. 5 and Eq. 6, in this engine's units).  With
     * ae_options.tier_stats, `candidates` counts the DP cells the trie levels evaluated (the
     * diagonal and vertical-gap slots of every (child, parent entry) pair), `pruned_nonpos`
     * those dropped with a value <= 0 (Theorem 2 (i)) and `pruned_reach` those dropped with
     * 0 < value <= thr(j), unable to reach H (Theorem 2 (ii)); the filtering ratio is
     * (pruned_nonpos + pruned_reach) / candidates.  `reused` (always counted) is the number of
     * entries of rows handed to the text-position sweep that a row already walking through
     * the same text position absorbed -- computed once for both from there on; the reusing
     * ratio is reused / (reused + entries). */
    int64_t candidates, pruned_nonpos, pruned_reach;
    int64_t reused;
    int64_t reroutes;         /* engine batches whose frontier left the int16x2 route for int32 (a
                                 state could pass the int16 range; nothing is recomputed) */
    int64_t leaf_wide_walks;  /* walks of the text-position sweep continued on a thread block
                                 (ae_options.leaf_wide_rows) */
} ae_stats;

/* Engine knobs (NULL = defaults).  None of them changes the result set. */
typedef struct {
    int32_t qprefix_seed;   /* 1: start at depth q-1 from the query's (q-1)-grams (Theorem 3); 0: root */
    int32_t leaf_segment;   /* injected rows per sweep task (0 = chosen from the load) */
    int64_t item_columns;   /* query columns per work item (seed range) */
    int64_t batch_columns;  /* query columns processed per batch */
    int32_t leaf_capacity;  /* initial per-task row capacity of the sweep, in entries */
    int32_t profile;        /* 1: time kernel groups with CUDA events (ae_stats.ms_k_*) */
    int32_t leaf_delay;     /* levels (0-14) a single-occurrence trie node keeps expanding in the
                               trie walk before its row moves to the text-position sweep */
    int32_t int16_limit;    /* trie rows are stored as int16x2 (M, G_a) pairs while depth * g_max
                               stays <= this (<= 32000; 0 = int32 throughout); past it the
                               frontier is unpacked to int32 and the walk continues exactly */
    const int64_t *hint_hits; /* host, one per query, or NULL: expected hit records of the query's
                                 text-position sweep (e.g. from ae_mlp_forward); each batch's sweep
                                 hit buffer is then sized from the hints of its queries instead of
                                 from the previous searches on the stream.  A low hint costs one
                                 rerun of the sweep, never a result */
    int32_t tier_stats;       /* 1: count trie entries by cost tier into ae_stats.entries_tier
                                 (a few instructions per entry); 0: leave them 0 */
    int64_t workspace_limit;  /* > 0: cap on the device bytes of the stream's workspace; a batch
                                 that would grow it further is searched as two halves (as after
                                 a failed device allocation; ae_stats.batch_splits); a single
                                 query column that does not fit gives AE_ENOMEM.  0: no cap */
    int32_t general_rows;     /* 1: compute every trie level with the general row kernel (any alphabet,
                                 one lane per (child, parent entry)) instead of the DNA int16x2 kernel
                                 (one lane per parent entry, all children); the results are the same */
    int32_t qprefix_domination; /* 1 (default): with q-prefix seeding, drop the forks that Lemma 1's
                                 domination proves redundant -- a seed gram every occurrence of which
                                 in T is preceded by the query letter before the fork's start (a table
                                 of the letters preceding each gram is built once per index and seed
                                 depth); 0: keep every fork.  The results are the same */
    int32_t row_layout;       /* DNA int16x2 kernel: 0 (default) chooses per trie level, 1 walks each
                                 parent row in one lane per (node, child), 2 spreads each row over the
                                 lanes one entry per lane, 3 gives each node a whole thread block.
                                 The results are the same */
    /* A search split over ranks or devices: with fork_parts = R > 1 the search keeps only part
     * fork_part (0 <= fork_part < R) of the forks -- the seed subtrees whose gram hashes to the
     * part (q-prefix seeding), or the start columns j with j % R == fork_part (walks from the
     * root).  The R parts together cover every fork once, so the per-cell maximum over their
     * results (ae_hits_merge) is the full search's result set; one part alone may miss a result
     * or report it with a lower score.  Defaults: 1 and 0 (the whole search). */
    int32_t fork_parts;
    int32_t fork_part;
    int32_t leaf_wide_rows;   /* a walk of the text-position sweep whose row grows past this many
                                 entries continues on a whole thread block (each step spread over
                                 its threads) instead of one warp; 0: never.  Default 128.  The
                                 results are the same */
} ae_options;

/* Fill *opt with the defaults: qprefix_seed 1, leaf_segment 0, item_columns
 * 2^24, batch_columns 2^20, leaf_capacity 4096, profile 0, leaf_delay 8,
 * int16_limit 32000, hint_hits NULL, tier_stats 0, workspace_limit 0,
 * general_rows 0, qprefix_domination 1, row_layout 0, fork_parts 1,
 * fork_part 0, leaf_wide_rows 128. */
void ae_options_default(ae_options *opt);

/* Build an index of text[0..n) (host ASCII) for `alphabet` (AE_DNA or
 * AE_PROTEIN): the suffix array of the reversed text followed by a sentinel,
 * its BWT packed into occurrence blocks (2-bit symbols for DNA, 5 bit-planes
 * for protein) with sampled ranks, the text-end array (entry h = end position
 * in T of the substrings whose reverse prefixes suffix h), and the forward
 * text (Section 2.3 and Section 5 (1)-(3)).  The suffix array is built on the
 * current CUDA device (ae_suffix_array_device, about 33 bytes of device memory
 * per letter while it runs).  The occurrence blocks are filled from it on the
 * host, and the index is then copied once to the device.
 * Errors: AE_EINVAL (n < 1, unknown letter, bad alphabet), AE_EUNSUPPORTED
 * (n >= 2^31 - 1), AE_ENOMEM, AE_ECUDA. */
ae_status ae_index_build(const uint8_t *text, int64_t n, int32_t alphabet, ae_index **out);

/* Build an index of a collection of sequences (Section 2.3: a database of
 * several sequences searched as one text).  text[0..n) (host ASCII) holds the
 * nseq sequences back to back; starts[0..nseq) (host) are their first
 * positions, starts[0] = 0, non-decreasing, <= n (sequence k is
 * text[starts[k] .. starts[k+1]), the last one ends at n; empty sequences are
 * allowed).  The sequences are indexed joined by a separator that sorts below
 * every letter and matches nothing, so no result's alignment spans two
 * sequences; result positions (ae_hit.text_end) are positions in text, i.e.
 * in the sequences back to back.  Otherwise as ae_index_build, whose index of
 * a single sequence this equals in results.
 * Errors: AE_EINVAL (n < 1, bad starts, unknown letter, bad alphabet),
 * AE_EUNSUPPORTED (n + nseq >= 2^31 - 1), AE_ENOMEM, AE_ECUDA. */
ae_status ae_index_build_collection(const uint8_t *text, int64_t n, const int64_t *starts, int32_t nseq,
                                   int32_t alphabet, ae_index **out);

/* Write / read an index file (versioned header + checksum).  Load copies to
 * the current device.  Errors: AE_EIO, AE_ENOMEM, AE_ECUDA. */
ae_status ae_index_save(const ae_index *idx, const char *path);
ae_status ae_index_load(const char *path, ae_index **out);

/* Release the index and its device memory (NULL is ignored). */
void ae_index_free(ae_index *idx);

/* Text length, alphabet and device bytes held by the index. */
ae_status ae_index_info(const ae_index *idx, int64_t *n, int32_t *alphabet, int64_t *device_bytes);

/* Search nq host queries with per-query thresholds H[k] >= 1 (host array).
 * On success *hits is one library-allocated host array holding every result,
 * grouped by query in input order and sorted by (text_end, query_end) inside
 * a group; counts[k] (host, nq entries) is the number of results of query k.
 * Free *hits with ae_hits_free.  stream is a cudaStream_t (NULL = the legacy
 * default stream); the call returns after the results are on the host.
 * Results past 32 MiB are copied out by up to 8 host threads through pinned
 * chunks (8 MiB, two per thread, kept with the stream's workspace); the call
 * returns after those threads have finished.
 * Errors: AE_EINVAL, AE_ENOMEM, AE_ECUDA, AE_EUNSUPPORTED. */
ae_status ae_search(const ae_index *idx, const ae_query *queries, int32_t nq,
                    const ae_scoring *scoring, const int32_t *H, const ae_options *opt,
                    ae_hit **hits, int64_t *counts, void *stream);

void ae_hits_free(ae_hit *hits);

/* Same search with device-resident input and output.  d_seq (device) holds the
 * nq queries' ASCII letters back to back; offsets (host, nq+1 entries) delimit
 * query k as d_seq[offsets[k] .. offsets[k+1]).  Results are written to d_hits
 * (device, capacity entries) in the order ae_search uses, and counts (host, nq)
 * receives the per-query result counts.  If the total exceeds capacity nothing
 * is written to d_hits, counts still holds the required sizes, and the call
 * returns AE_EOVERFLOW.  Working memory is allocated by the library and kept
 * on the index between calls. */
ae_status ae_search_device(const ae_index *idx, const uint8_t *d_seq, const int64_t *offsets,
                           int32_t nq, const ae_scoring *scoring, const int32_t *H,
                           const ae_options *opt, ae_hit *d_hits, int64_t capacity,
                           int64_t *counts, void *stream);

/* The search of ae_search_device for callers that cannot allocate device
 * memory: a process whose device memory is already handed out to another
 * allocator (a framework's caching pool, a fixed reservation made at start-up)
 * and that must not take more behind that allocator's back.  It calls no
 * cudaMalloc, cudaFree, cudaMallocHost or other device allocator: every
 * working buffer is carved from one fixed 64 MiB array in the library's device
 * image, which each GPU that loads the library keeps until the process exits.
 * The paper has no counterpart; the arguments, result order and AE_EOVERFLOW
 * behaviour are those of ae_search_device.
 * Limits: at most 65,536 query letters in total and 4,096 queries per call,
 * and the search's working set must fit the array (rows of the
 * text-position sweep start at no more than 256 entries and may grow
 * fourfold up to 1,024); beyond that the call returns AE_EUNSUPPORTED and
 * writes nothing to d_hits.
 * The call synchronises `stream` while it runs (it reads each trie level's
 * sizes back to the host).
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current.  All calls on a device
 * share the array, which keeps the previous call's contents (the search
 * initialises everything it reads); calls on one device are serialised by the
 * library and each returns only after all of its device work has finished --
 * also when it fails part-way -- so their device work never overlaps: work
 * that did overlap on the same array would race. */
ae_status ae_search_device_static(const ae_index *idx, const uint8_t *d_seq, const int64_t *offsets,
                                  int32_t nq, const ae_scoring *scoring, const int32_t *H,
                                  const ae_options *opt, ae_hit *d_hits, int64_t capacity,
                                  int64_t *counts, void *stream);

/* Per-cell maximum over the results of several partial searches (Algorithm 1
 * lines 6-10, the maximum over all forks of a cell, when the forks were split
 * over searches with ae_options.fork_parts, e.g. over ranks or devices).
 * d_hits (device, n records) holds results of queries 0..nq-1, d_qid (device,
 * n int32) the query of each record; positions are < text_len and query ends
 * < max_query_len.  d_out (device, capacity n) receives one record per
 * distinct (query, text end, query end) with the largest score, grouped by
 * query and sorted by (text_end, query_end) -- the order of ae_search --
 * counts (host, nq) the records per query and *total their number.  The call
 * allocates and frees its sort buffers and returns after `stream` finished.
 * The paper has no counterpart (its search runs on one machine).
 * Errors: AE_EINVAL, AE_EUNSUPPORTED (keys wider than 64 bits), AE_ENOMEM,
 * AE_ECUDA. */
ae_status ae_hits_merge(const ae_hit *d_hits, const int32_t *d_qid, int64_t n, int32_t nq, int64_t text_len,
                        int64_t max_query_len, ae_hit *d_out, int64_t *counts, int64_t *total, void *stream);

/* Working memory.  ae_search and ae_search_device keep one workspace per
 * (index, stream): device buffers that only grow, reused by the next search on
 * that stream.  Searches on different streams run concurrently (an index is
 * shareable across threads); searches on one stream are serialised by the
 * library.  ae_workspace_info reports the device bytes held by the workspace
 * of `stream` (0 if it has none) and by all workspaces of the process;
 * ae_workspace_release waits for that stream's running search, then frees its
 * workspace (the next search on the stream starts a new one).
 * Errors: AE_EINVAL (idx NULL). */
ae_status ae_workspace_info(const ae_index *idx, void *stream, int64_t *bytes, int64_t *process_bytes);
ae_status ae_workspace_release(ae_index *idx, void *stream);

/* Counters of the calling thread's last search. */
ae_status ae_last_stats(ae_stats *out);

/* Suffix arrays, exposed for tests and for callers that build their own
 * indexes. */

/* Suffix array of codes[0..n) followed by a sentinel smaller than every code
 * (so sa has n+1 entries and sa[0] = n).  codes are in [0, sigma).  Built on
 * the host with induced sorting (SA-IS, Nong, Zhang & Chan 2009).  Host
 * memory.  The index build uses the device version below. */
ae_status ae_suffix_array(const uint8_t *codes, int64_t n, int32_t sigma, int32_t *sa);

/* The same suffix array computed on the device, as ae_index_build does for
 * the reversed text (Section 2.3; Section 5 (1)).  s = d_codes[0..n), or with
 * reversed != 0 the codes read backwards (s[k] = d_codes[n-1-k]); d_sa[0..n]
 * receives the start positions of the suffixes of s followed by a sentinel
 * smaller than every code, in lexicographic order (d_sa[0] = n).
 * Method: prefix doubling (Manber & Myers 1993).  Each suffix's first key
 * packs its first 64/b letters (b bits per letter value and the sentinel),
 * and a stable LSD radix sort groups equal keys.  The group index becomes the
 * rank, and the next key (rank of i, rank of i + h) orders by twice as many
 * letters.  Rounds stop when every rank is distinct.
 * d_codes and d_sa are device memory: codes in [0, sigma), 1 <= sigma <= 255,
 * 0 <= n < 2^31 - 2.  The call allocates and frees about 33 bytes of device
 * memory per letter, and returns once `stream` (NULL = the legacy default
 * stream) has finished its work.
 * Errors: AE_EINVAL (NULL pointer, sigma out of range, a code >= sigma),
 * AE_EUNSUPPORTED (n too large), AE_ENOMEM, AE_ECUDA. */
ae_status ae_suffix_array_device(const uint8_t *d_codes, int64_t n, int32_t sigma, int32_t reversed, int32_t *d_sa,
                                 void *stream);

/* For a query of length m over `alphabet`: q of Eq. 2 (0 with a matrix), the
 * depth the trie walk starts at, and L_max of Eq. 1 (with the largest matrix
 * entry in place of s_a when a matrix is given).  Outputs may be NULL. */
ae_status ae_plan(int64_t m, int32_t alphabet, const ae_scoring *scoring, int32_t H,
                  int32_t *q, int32_t *seed_depth, int64_t *L_max);

/* Human-readable text of a status code (static storage). */
const char *ae_strerror(int32_t status);

#ifdef __cplusplus
}
#endif

#endif /* AE_H */
