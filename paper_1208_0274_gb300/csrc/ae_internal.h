// Internal declarations shared by the host index builder, the kernels and the
// engine of libae.  Nothing here is part of the public ABI (include/ae.h).
#pragma once

#include <stdint.h>
#include <stddef.h>

#include "ae.h"

#ifdef __CUDACC__
#define AE_HD __host__ __device__
#else
#define AE_HD
#endif

// Value of a pruned ("meaningless", Theorem 2) DP state.  Far below any live
// score, far enough above INT32_MIN that adding a few gap charges cannot wrap.
#define AE_NEG (-(1 << 28))
// Key of "no candidate" in the horizontal-gap max-plus scan.
#define AE_KNEG (-(1 << 30))

#define AE_MAX_SIGMA 20

// ---------------------------------------------------------------- index layout
// DNA: one 32-byte block per 64 BWT rows: 4 x u32 occurrence counts of A,C,G,T
// in rows [0, 64b) (the sentinel not counted), then 4 x u32 holding the 64
// rows' 2-bit codes (row r of the block in bits 2*(r%16) of word r/16; the
// sentinel row stores code 0).
// Protein: one 128-byte block per 64 rows: 20 x u32 counts, 2 x u32 pad, then
// 5 x u64 bit-planes (bit r of plane t = bit t of row r's 5-bit code).
#define AE_DNA_BLOCK_WORDS 8
#define AE_PROT_BLOCK_WORDS 32
#define AE_ROWS_PER_BLOCK 64

// Collections (several sequences indexed as one text, Section 2.3): the BWT
// is that of the sequences joined by a separator that sorts below every
// letter.  A separator row stores letter code 0 in its block and is flagged in
// `sep`: 4 words per occurrence block, the number of separator rows before the
// block and a 64-bit mask of the block's separator rows (low word first); the
// block's letter counts leave separators out, and Occ(0, k) subtracts the
// flagged rows of k's own block.  Positions (tend, text, results) are those of the
// sequences joined without separators; `ends` has bit p set where position p is
// the last letter of a sequence, which no alignment may cross.
#define AE_SEP_BLOCK_WORDS 4

struct IndexView {
    const uint32_t *occ;    // blocks
    const int32_t *tend;    // per BWT row: end position in T of its substrings (-1 = sentinel row)
    const uint8_t *text;    // forward text, letter codes
    int64_t n;              // text length (letters, separators not counted)
    int64_t dollar_row;     // BWT row holding the sentinel
    uint32_t C[AE_MAX_SIGMA + 1];  // C[c] = 1 + separators + number of letters < c; C[sigma] = rows
    int32_t sigma;
    int32_t alphabet;
    int64_t rows;           // BWT rows: n + separators + 1
    const uint32_t *sep;    // collections: separator rows per block (NULL for one sequence)
    const uint32_t *ends;   // collections: sequence-end bitmap over text positions (NULL for one sequence)
};

struct ScoreView {
    int32_t sa, sb, sg, ss;    // <s_a, s_b, s_g, s_s>
    int32_t use_matrix;
    int32_t gmax;              // largest gain of one query column (s_a or max matrix entry)
    int8_t mat[AE_MAX_SIGMA * AE_MAX_SIGMA];   // delta(text letter, query letter)
};

// Per-query arrays of one search (device pointers).
struct QueryView {
    const uint8_t *codes;      // all queries' letter codes back to back
    const int64_t *off;        // start of query k in codes
    const int32_t *m;          // length of query k
    const int32_t *H;          // threshold of query k
};

// A work item: the forks of query `qid` whose first column lies in [c0, c1).
struct WorkItem {
    int32_t qid;
    int32_t c0, c1;
    int32_t pad;
};

// A frontier node: SA range [lo, hi) of the reversed prefix at this depth,
// its row stored at [off, off + cnt) of the level arena.  cnt == ROOT_ROW
// marks the implicit depth-0 row (M(0, j) = 0 for the item's columns); `item`
// is the work item of a root node and the query id of every other node.
struct Node {
    uint32_t lo, hi;
    int32_t item;
    uint32_t cnt;
    uint64_t off;
};
#define AE_ROOT_ROW 0xFFFFFFFFu

// A row handed from the trie walk to the text-position sweep: the node became
// a single occurrence ending at text position `e`.
struct Inject {
    int32_t qid;
    int32_t e;
    uint32_t cnt;
    uint32_t pad;
    uint64_t off;
};

// A result before the per-cell maximum, as a range of BWT rows (trie nodes
// with several occurrences).
struct RangeHit {
    uint32_t lo, hi;
    int32_t qid;
    int32_t j;
    int32_t score;
    int32_t pad;
};

// Device counters of one search (all atomics, summed).
struct DevStats {
    unsigned long long nodes, leaf_rows, entries, tier[3], raw_hits;
    unsigned long long leaf_overflow, hit_overflow;
    unsigned long long entries_leaf;
    unsigned long long leaf_max_steps, leaf_max_width;
    unsigned long long leaf_max_cycles;   // longest sweep task (SM clock cycles)
    unsigned long long dominated;         // seed entries dropped by q-prefix domination (Lemma 1)
    unsigned long long reused;            // sweep: injected entries absorbed by a walked row at their position
    unsigned long long cand, pruned_nonpos, pruned_reach;   // tier_stats: slot candidates of the trie
                                                            // levels and those the filters dropped
    unsigned long long pad;
};

// ---------------------------------------------------------------- host index
struct HostIndex {
    int32_t alphabet, sigma;
    int64_t n;
    int64_t dollar_row;
    uint32_t C[AE_MAX_SIGMA + 1];
    int64_t nblocks;
    int32_t block_words;
    uint32_t *occ;     // nblocks * block_words
    int32_t *tend;     // rows
    uint8_t *text;     // n codes
    int64_t rows;      // BWT rows (n + 1 + separators)
    int32_t nseq;      // sequences of a collection (0: a single text)
    uint32_t *sep;     // collections: nblocks * AE_SEP_BLOCK_WORDS
    uint32_t *ends;    // collections: (n + 31) / 32 words
};

int ae_alphabet_sigma(int32_t alphabet);
int ae_encode_letters(const uint8_t *ascii, int64_t n, int32_t alphabet, uint8_t *codes);
void ae_letter_lut(int32_t alphabet, uint8_t lut[256]);
ae_status ae_host_index_fill(const uint8_t *codes, int64_t n, int32_t alphabet, const int32_t *sa, HostIndex *out);
// The index of a collection: codes[0..n) are the sequences back to back,
// starts[0..nseq) their first positions (starts[0] = 0, non-decreasing); sa is
// the suffix array of the reversed joined text (nseq - 1 separators of code 0,
// letters shifted up by one) followed by the sentinel.
ae_status ae_host_index_fill_collection(const uint8_t *codes, int64_t n, const int64_t *starts, int32_t nseq,
                                        int32_t alphabet, const int32_t *sa, HostIndex *out);
void ae_host_index_free(HostIndex *h);
ae_status ae_host_index_save(const HostIndex *h, const char *path);
ae_status ae_host_index_load(const char *path, HostIndex *h);

// Device view of a built index (pointers into the index's device memory).
const IndexView *ae_index_view(const ae_index *idx);
