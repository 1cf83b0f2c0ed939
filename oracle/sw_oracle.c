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
 * similarity is at least H (Algorithm 1, line 11).
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
 * Arithmetic is int64, rows are kept two at a time, one thread.
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
