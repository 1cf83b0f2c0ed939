/*
 * CPU oracle for exact local-alignment search — TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load this library. The GPU search path never calls it.
 *
 * What it computes (Section 2.1, "Local alignment problem"; Table 1, A(i,j)):
 * for every text end i and query end j, the largest similarity between a
 * substring T[x..i] and a substring P[y..j], where the similarity of two strings
 * is the best score of a global alignment of them under the scheme
 * <s_a, s_b, s_g, s_s> (a run of r gap letters scores s_g + r*s_s).  For a
 * threshold H >= 1 the reported results are the cells whose largest
 * similarity is at least H (the hit report of Algorithm 1).
 *
 * The value is the textbook affine-gap Smith-Waterman cell (Gotoh's three
 * states), written out over the full n x m matrix with no index and no
 * filter:
 *     E(i,j) = max(E(i-1,j) + s_s, V(i-1,j) + s_g + s_s)    text letter vs gap
 *     F(i,j) = max(F(i,j-1) + s_s, V(i,j-1) + s_g + s_s)    query letter vs gap
 *     V(i,j) = max(0, V(i-1,j-1) + delta(T[i],P[j]), E(i,j), F(i,j))
 * with V = 0 and E = F = -inf on row 0 / column 0.  The 0 term lets an
 * alignment start at any cell; every positive V(i,j) is the largest
 * similarity above (the 0 is only taken when all candidates are <= 0, which
 * never meets H >= 1).  delta(a,b) is looked up in a sigma x sigma table
 * (s_a on the diagonal and s_b elsewhere for the paper's schemes).
 *
 * Arithmetic is int64, rows are kept two at a time; ae_oracle_sw_hits runs
 * on one thread, ae_oracle_sw_hits_mt (end of file) on several.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_NEG (INT64_MIN / 4)

static inline int64_t max2(int64_t a, int64_t b) { return a > b ? a : b; }

/* Local-alignment cell values >= H.
 *   T[0..n), P[0..m): letter codes in [0, sigma).
 *   subst: sigma*sigma row-major, subst[a*sigma + b] = delta(text a, query b).
 *   Rows i < row_lo are computed but not reported (window checks).
 *   Hits are written as 0-based inclusive ends (out_i, out_j) and score out_s,
 *   in row-major order, at most cap of them; the return value is the total
 *   number of hits (> cap means the buffers were too small), or -1 on a bad
 *   argument or allocation failure. */
int64_t ae_oracle_sw_hits(const uint8_t *T, int64_t n, const uint8_t *P, int64_t m,
                          const int32_t *subst, int32_t sigma,
                          int32_t gap_open, int32_t gap_extend, int32_t H,
                          int64_t row_lo,
                          int64_t *out_i, int32_t *out_j, int32_t *out_s, int64_t cap)
{
    if (n < 0 || m < 0 || sigma <= 0 || !subst) return -1;
    if (n == 0 || m == 0) return 0;
    int64_t *Vp = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m + 1));
    int64_t *Vc = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m + 1));
    int64_t *E = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m + 1));
    if (!Vp || !Vc || !E) { free(Vp); free(Vc); free(E); return -1; }
    const int64_t open_ext = (int64_t)gap_open + gap_extend;
    for (int64_t j = 0; j <= m; ++j) { Vp[j] = 0; E[j] = ORACLE_NEG; }
    int64_t count = 0;
    for (int64_t i = 1; i <= n; ++i) {
        const int32_t *row = subst + (int64_t)T[i - 1] * sigma;
        int64_t F = ORACLE_NEG;
        Vc[0] = 0;
        for (int64_t j = 1; j <= m; ++j) {
            E[j] = max2(E[j] + gap_extend, Vp[j] + open_ext);
            F = max2(F + gap_extend, Vc[j - 1] + open_ext);
            int64_t v = Vp[j - 1] + row[P[j - 1]];
            v = max2(v, E[j]);
            v = max2(v, F);
            v = max2(v, 0);
            Vc[j] = v;
            if (v >= H && i - 1 >= row_lo) {
                if (count < cap) {
                    out_i[count] = i - 1;
                    out_j[count] = (int32_t)(j - 1);
                    out_s[count] = (int32_t)v;
                }
                ++count;
            }
        }
        int64_t *t = Vp; Vp = Vc; Vc = t;
    }
    free(Vp); free(Vc); free(E);
    return count;
}

/* The full V matrix (n x m, row-major, int64) for small property tests. */
int ae_oracle_sw_matrix(const uint8_t *T, int64_t n, const uint8_t *P, int64_t m,
                        const int32_t *subst, int32_t sigma,
                        int32_t gap_open, int32_t gap_extend, int64_t *V)
{
    if (n < 0 || m < 0 || sigma <= 0 || !subst) return -1;
    int64_t *Vp = (int64_t *)calloc((size_t)(m + 1), sizeof(int64_t));
    int64_t *Vc = (int64_t *)calloc((size_t)(m + 1), sizeof(int64_t));
    int64_t *E = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m + 1));
    if (!Vp || !Vc || !E) { free(Vp); free(Vc); free(E); return -1; }
    const int64_t open_ext = (int64_t)gap_open + gap_extend;
    for (int64_t j = 0; j <= m; ++j) E[j] = ORACLE_NEG;
    for (int64_t i = 1; i <= n; ++i) {
        const int32_t *row = subst + (int64_t)T[i - 1] * sigma;
        int64_t F = ORACLE_NEG;
        Vc[0] = 0;
        for (int64_t j = 1; j <= m; ++j) {
            E[j] = max2(E[j] + gap_extend, Vp[j] + open_ext);
            F = max2(F + gap_extend, Vc[j - 1] + open_ext);
            int64_t v = max2(max2(Vp[j - 1] + row[P[j - 1]], E[j]), max2(F, 0));
            Vc[j] = v;
            V[(i - 1) * m + (j - 1)] = v;
        }
        int64_t *t = Vp; Vp = Vc; Vc = t;
    }
    free(Vp); free(Vc); free(E);
    return 0;
}

/* Suffix array (Section 2.3): the start positions of the suffixes of
 * codes[0..n) followed by a sentinel smaller than every letter, listed in
 * lexicographic order of the suffixes.  Written as that definition: qsort of
 * the n + 1 start positions with a comparator that compares two suffixes
 * letter by letter (memcmp over the letters shifted up by one, the sentinel
 * stored as 0).  The sentinel occurs once, so two different suffixes never
 * compare equal.  codes are < 255.  Returns 0, or -1 when out of memory.
 * Not reentrant (the comparator reads the text through file-level state). */
static const uint8_t *sa_text;
static int64_t sa_len;

static int sa_compare(const void *x, const void *y) {
    int64_t a = *(const int32_t *)x, b = *(const int32_t *)y;
    /* the shorter suffix has sa_len - max(a, b) letters, its sentinel last */
    int64_t len = sa_len - (a > b ? a : b);
    int c = memcmp(sa_text + a, sa_text + b, (size_t)len);
    if (c) return c;
    return (a > b) - (a < b);   /* not reached: the sentinel differs */
}

int ae_oracle_suffix_array(const uint8_t *codes, int64_t n, int32_t *sa) {
    uint8_t *s = (uint8_t *)malloc((size_t)n + 1);
    if (!s) return -1;
    for (int64_t i = 0; i < n; ++i) s[i] = (uint8_t)(codes[i] + 1);
    s[n] = 0;
    for (int64_t i = 0; i <= n; ++i) sa[i] = (int32_t)i;
    sa_text = s;
    sa_len = n + 1;
    qsort(sa, (size_t)n + 1, sizeof(int32_t), sa_compare);
    free(s);
    return 0;
}

/* ---------------------------------------------------------------- all cores
 *
 * ae_oracle_sw_hits_mt: exactly the values of ae_oracle_sw_hits (the same
 * recurrence, int64), spread over `threads` host threads.  The query columns
 * are cut into one stripe per thread; thread t computes its stripe a block of
 * OR_ROWS text rows at a time, after thread t-1 has finished the same rows of
 * the stripe to its left (a wavefront over (row block, stripe) tiles).  The
 * only values that cross a stripe edge are V and F of the edge column for
 * each row, handed over through a small ring of row blocks.  Hits are kept
 * per thread and merged into the row-major order of ae_oracle_sw_hits.
 */
#include <pthread.h>
#include <sched.h>
#include <stdatomic.h>

#define OR_ROWS 256
#define OR_RING 8

typedef struct {
    /* shared problem */
    const uint8_t *T, *P;
    int64_t n, m;
    const int32_t *subst;
    int32_t sigma, gap_extend, H;
    int64_t open_ext, row_lo;
    int nthreads;
    /* per thread */
    int64_t *c0;                  /* stripe t = columns [c0[t], c0[t+1]) (1-based j in (c0, c1]) */
    atomic_llong *done;           /* rows finished by thread t */
    int64_t *edgeV, *edgeF;       /* ring: thread t's right-edge V and F, [t][slot][row in block] */
    int64_t **hi; int32_t **hj, **hs;
    int64_t *hcount, *hcap;
    int *fail;
    atomic_int abort_all;         /* set when not every thread could be started */
} or_job;

typedef struct { or_job *job; int t; } or_arg;

static void or_wait(or_job *J, atomic_llong *x, int64_t want) {
    while (atomic_load_explicit(x, memory_order_acquire) < want) {
        if (atomic_load_explicit(&J->abort_all, memory_order_relaxed)) return;
        sched_yield();
    }
}

static int or_push(or_job *J, int t, int64_t i, int32_t j, int32_t s) {
    if (J->hcount[t] == J->hcap[t]) {
        int64_t nc = J->hcap[t] ? 2 * J->hcap[t] : 4096;
        int64_t *a = (int64_t *)realloc(J->hi[t], sizeof(int64_t) * (size_t)nc);
        if (!a) return -1;
        J->hi[t] = a;
        int32_t *b = (int32_t *)realloc(J->hj[t], sizeof(int32_t) * (size_t)nc);
        if (!b) return -1;
        J->hj[t] = b;
        int32_t *c = (int32_t *)realloc(J->hs[t], sizeof(int32_t) * (size_t)nc);
        if (!c) return -1;
        J->hs[t] = c;
        J->hcap[t] = nc;
    }
    J->hi[t][J->hcount[t]] = i;
    J->hj[t][J->hcount[t]] = j;
    J->hs[t][J->hcount[t]] = s;
    J->hcount[t]++;
    return 0;
}

static void *or_worker(void *p) {
    or_arg *A = (or_arg *)p;
    or_job *J = A->job;
    const int t = A->t;
    const int64_t a = J->c0[t], b = J->c0[t + 1], w = b - a;   /* columns a+1 .. b */
    int64_t *Vp = (int64_t *)malloc(sizeof(int64_t) * (size_t)(w + 1));
    int64_t *Vc = (int64_t *)malloc(sizeof(int64_t) * (size_t)(w + 1));
    int64_t *E = (int64_t *)malloc(sizeof(int64_t) * (size_t)(w + 1));
    int bad = !Vp || !Vc || !E;
    if (!bad) for (int64_t k = 0; k <= w; ++k) { Vp[k] = 0; E[k] = ORACLE_NEG; }
    int64_t left_prev = 0;   /* V(i-1, a): the left neighbour's edge value of the previous row */
    for (int64_t r0 = 0; r0 < J->n; r0 += OR_ROWS) {
        const int64_t r1 = r0 + OR_ROWS < J->n ? r0 + OR_ROWS : J->n;
        const int64_t blk = r0 / OR_ROWS, slot = blk % OR_RING;
        if (t > 0) or_wait(J, &J->done[t - 1], r1);                 /* left stripe has these rows */
        if (t + 1 < J->nthreads && blk >= OR_RING)                  /* right stripe consumed the slot */
            or_wait(J, &J->done[t + 1], (blk - OR_RING + 1) * OR_ROWS);
        if (atomic_load_explicit(&J->abort_all, memory_order_relaxed)) break;
        const int64_t *lV = t > 0 ? J->edgeV + ((int64_t)(t - 1) * OR_RING + slot) * OR_ROWS : NULL;
        const int64_t *lF = t > 0 ? J->edgeF + ((int64_t)(t - 1) * OR_RING + slot) * OR_ROWS : NULL;
        int64_t *oV = J->edgeV + ((int64_t)t * OR_RING + slot) * OR_ROWS;
        int64_t *oF = J->edgeF + ((int64_t)t * OR_RING + slot) * OR_ROWS;
        const int64_t ge = J->gap_extend, oe = J->open_ext, H = J->H, row_lo = J->row_lo;
        const uint8_t *Pa = J->P + a;
        for (int64_t i = r0 + 1; i <= r1 && !bad; ++i) {
            const int32_t *row = J->subst + (int64_t)J->T[i - 1] * J->sigma;
            /* column a of row i (0 at the matrix edge) and its F */
            int64_t F = t > 0 ? lF[i - 1 - r0] : ORACLE_NEG;
            Vc[0] = t > 0 ? lV[i - 1 - r0] : 0;
            Vp[0] = left_prev;
            for (int64_t k = 1; k <= w; ++k) {
                E[k] = max2(E[k] + ge, Vp[k] + oe);
                F = max2(F + ge, Vc[k - 1] + oe);
                int64_t v = Vp[k - 1] + row[Pa[k - 1]];
                v = max2(v, E[k]);
                v = max2(v, F);
                v = max2(v, 0);
                Vc[k] = v;
                if (v >= H && i - 1 >= row_lo && or_push(J, t, i - 1, (int32_t)(a + k - 1), (int32_t)v)) {
                    bad = 1;
                    break;
                }
            }
            oV[i - 1 - r0] = Vc[w];
            oF[i - 1 - r0] = F;
            left_prev = Vc[0];
            int64_t *tmp = Vp; Vp = Vc; Vc = tmp;
        }
        if (bad) { *J->fail = 1; }
        atomic_store_explicit(&J->done[t], r1, memory_order_release);
    }
    free(Vp); free(Vc); free(E);
    return NULL;
}

/* As ae_oracle_sw_hits, on `threads` host threads (threads <= 0: 1).  Same
 * arguments, same results in the same order, same return convention. */
int64_t ae_oracle_sw_hits_mt(const uint8_t *T, int64_t n, const uint8_t *P, int64_t m,
                             const int32_t *subst, int32_t sigma,
                             int32_t gap_open, int32_t gap_extend, int32_t H,
                             int64_t row_lo, int32_t threads,
                             int64_t *out_i, int32_t *out_j, int32_t *out_s, int64_t cap)
{
    if (n < 0 || m < 0 || sigma <= 0 || !subst) return -1;
    if (n == 0 || m == 0) return 0;
    int nt = threads < 1 ? 1 : threads;
    if (nt > 256) nt = 256;
    if ((int64_t)nt > m) nt = (int)m;
    or_job J;
    memset(&J, 0, sizeof(J));
    J.T = T; J.P = P; J.n = n; J.m = m; J.subst = subst; J.sigma = sigma;
    J.gap_extend = gap_extend; J.H = H; J.open_ext = (int64_t)gap_open + gap_extend; J.row_lo = row_lo;
    J.nthreads = nt;
    int fail = 0;
    J.fail = &fail;
    J.c0 = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nt + 1));
    J.done = (atomic_llong *)malloc(sizeof(atomic_llong) * (size_t)nt);
    J.edgeV = (int64_t *)malloc(sizeof(int64_t) * (size_t)nt * OR_RING * OR_ROWS);
    J.edgeF = (int64_t *)malloc(sizeof(int64_t) * (size_t)nt * OR_RING * OR_ROWS);
    J.hi = (int64_t **)calloc((size_t)nt, sizeof(int64_t *));
    J.hj = (int32_t **)calloc((size_t)nt, sizeof(int32_t *));
    J.hs = (int32_t **)calloc((size_t)nt, sizeof(int32_t *));
    J.hcount = (int64_t *)calloc((size_t)nt, sizeof(int64_t));
    J.hcap = (int64_t *)calloc((size_t)nt, sizeof(int64_t));
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nt);
    or_arg *args = (or_arg *)malloc(sizeof(or_arg) * (size_t)nt);
    int64_t result = -1;
    if (J.c0 && J.done && J.edgeV && J.edgeF && J.hi && J.hj && J.hs && J.hcount && J.hcap && th && args) {
        for (int t = 0; t <= nt; ++t) J.c0[t] = m * t / nt;
        for (int t = 0; t < nt; ++t) atomic_init(&J.done[t], 0);
        atomic_init(&J.abort_all, 0);
        int started = 0;
        for (int t = 0; t < nt; ++t) {
            args[t].job = &J;
            args[t].t = t;
            if (pthread_create(&th[t], NULL, or_worker, &args[t]) != 0) break;
            ++started;
        }
        /* the stripes wait on their neighbours: without every thread the
         * wavefront cannot finish, so stop the others and report a failure */
        if (started < nt) {
            atomic_store(&J.abort_all, 1);
            fail = 1;
        }
        for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
        if (!fail) {
            /* row-major merge: rows ascending; inside a row, stripes left to right */
            int64_t total = 0;
            for (int t = 0; t < nt; ++t) total += J.hcount[t];
            int64_t *pos = (int64_t *)calloc((size_t)nt, sizeof(int64_t));
            if (pos) {
                int64_t k = 0;
                while (k < total) {
                    int64_t best = INT64_MAX;
                    for (int t = 0; t < nt; ++t)
                        if (pos[t] < J.hcount[t] && J.hi[t][pos[t]] < best) best = J.hi[t][pos[t]];
                    for (int t = 0; t < nt; ++t)
                        while (pos[t] < J.hcount[t] && J.hi[t][pos[t]] == best) {
                            if (k < cap) {
                                out_i[k] = best;
                                out_j[k] = J.hj[t][pos[t]];
                                out_s[k] = J.hs[t][pos[t]];
                            }
                            ++k;
                            ++pos[t];
                        }
                }
                free(pos);
                result = total;
            }
        }
    }
    if (J.hi) for (int t = 0; t < nt; ++t) free(J.hi[t]);
    if (J.hj) for (int t = 0; t < nt; ++t) free(J.hj[t]);
    if (J.hs) for (int t = 0; t < nt; ++t) free(J.hs[t]);
    free(J.hi); free(J.hj); free(J.hs); free(J.hcount); free(J.hcap);
    free(J.c0); free((void *)J.done); free(J.edgeV); free(J.edgeF); free(th); free(args);
    return result;
}

/* ---------------------------------------------------------------- restricted starts
 *
 * ae_oracle_sw_hits_starts: the largest similarity of alignments ending at
 * (i, j) that START at a query column y with allowed[y] != 0 (0-based), for
 * every cell, reported where it reaches H.  This is the result of the forks
 * one part of a split search owns; the maximum over a partition of the query
 * columns is the unrestricted value of ae_oracle_sw_hits at every cell >= H.
 * Written as the Gotoh recurrence without the floor at 0 (a floor would
 * re-start the alignment at any column): S = best restricted alignment ending
 * at the cell, E / F its vertical / horizontal gap states, and a fresh
 * alignment may begin only by pairing T[i] with an allowed P[j]:
 *     D(i,j) = delta(T[i],P[j]) + max(S(i-1,j-1), allowed[j] ? 0 : -inf)
 *     E(i,j) = max(E(i-1,j) + s_s, S(i-1,j) + s_g + s_s)
 *     F(i,j) = max(F(i,j-1) + s_s, S(i,j-1) + s_g + s_s)
 *     S(i,j) = max(D, E, F),   S = E = F = -inf outside the matrix.
 * (An optimal alignment never starts with a gap.)  Same arguments and
 * return convention as ae_oracle_sw_hits plus the allowed[0..m) mask.
 */
int64_t ae_oracle_sw_hits_starts(const uint8_t *T, int64_t n, const uint8_t *P, int64_t m,
                                 const int32_t *subst, int32_t sigma,
                                 int32_t gap_open, int32_t gap_extend, int32_t H,
                                 const uint8_t *allowed,
                                 int64_t *out_i, int32_t *out_j, int32_t *out_s, int64_t cap)
{
    if (n < 0 || m < 0 || sigma <= 0 || !subst || (m > 0 && !allowed)) return -1;
    if (n == 0 || m == 0) return 0;
    int64_t *Sp = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m + 1));
    int64_t *Sc = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m + 1));
    int64_t *E = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m + 1));
    if (!Sp || !Sc || !E) { free(Sp); free(Sc); free(E); return -1; }
    const int64_t open_ext = (int64_t)gap_open + gap_extend;
    for (int64_t j = 0; j <= m; ++j) { Sp[j] = ORACLE_NEG; E[j] = ORACLE_NEG; }
    int64_t count = 0;
    for (int64_t i = 1; i <= n; ++i) {
        const int32_t *row = subst + (int64_t)T[i - 1] * sigma;
        int64_t F = ORACLE_NEG;
        Sc[0] = ORACLE_NEG;
        for (int64_t j = 1; j <= m; ++j) {
            E[j] = max2(E[j] + gap_extend, Sp[j] + open_ext);
            F = max2(F + gap_extend, Sc[j - 1] + open_ext);
            int64_t prev = Sp[j - 1];
            if (allowed[j - 1]) prev = max2(prev, 0);
            int64_t v = prev + row[P[j - 1]];
            v = max2(v, E[j]);
            v = max2(v, F);
            if (v < ORACLE_NEG) v = ORACLE_NEG;   /* keep -inf from drifting */
            Sc[j] = v;
            if (v >= H) {
                if (count < cap) {
                    out_i[count] = i - 1;
                    out_j[count] = (int32_t)(j - 1);
                    out_s[count] = (int32_t)v;
                }
                ++count;
            }
        }
        int64_t *t = Sp; Sp = Sc; Sc = t;
    }
    free(Sp); free(Sc); free(E);
    return count;
}
