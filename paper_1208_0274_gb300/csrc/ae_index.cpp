// Host side of the FM index (Section 2.3 and Section 5): letter coding, a host
// suffix array by induced sorting (exported; the index build takes its suffix
// array from the device), the BWT packed into occurrence blocks from a suffix
// array of the reversed text, and the index file format.
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "ae_internal.h"

static const char kDNA[] = "ACGT";
static const char kProtein[] = "ARNDCQEGHILKMFPSTWYV";

int ae_alphabet_sigma(int32_t alphabet) {
    return alphabet == AE_DNA ? 4 : alphabet == AE_PROTEIN ? 20 : 0;
}

void ae_letter_lut(int32_t alphabet, uint8_t lut[256]) {
    memset(lut, 255, 256);
    const char *a = alphabet == AE_DNA ? kDNA : kProtein;
    int s = ae_alphabet_sigma(alphabet);
    for (int c = 0; c < s; ++c) lut[(uint8_t)a[c]] = (uint8_t)c;
}

// ASCII -> codes; returns 0 on success, -1 on a letter outside the alphabet.
int ae_encode_letters(const uint8_t *ascii, int64_t n, int32_t alphabet, uint8_t *codes) {
    uint8_t lut[256];
    ae_letter_lut(alphabet, lut);
    for (int64_t i = 0; i < n; ++i) {
        uint8_t c = lut[ascii[i]];
        if (c == 255) return -1;
        codes[i] = c;
    }
    return 0;
}

// ------------------------------------------------------------------ SA-IS
// Suffix array by induced sorting (Nong, Zhang & Chan, "Two efficient
// algorithms for linear time suffix array construction", 2009).  s[0..N) has
// letters in [0, K) and s[N-1] = 0 is a unique smallest sentinel.

namespace {

void bucket_bounds(const int32_t *s, int32_t N, int32_t K, int32_t *bkt, bool ends) {
    std::fill(bkt, bkt + K, 0);
    for (int32_t i = 0; i < N; ++i) ++bkt[s[i]];
    int32_t sum = 0;
    for (int32_t c = 0; c < K; ++c) {
        sum += bkt[c];
        bkt[c] = ends ? sum : sum - bkt[c];
    }
}

// Given the LMS suffixes already placed, induce the L-type suffixes from left
// to right and then the S-type suffixes from right to left.
void induce(const int32_t *s, int32_t *SA, const uint8_t *stype, int32_t N, int32_t K, int32_t *bkt) {
    bucket_bounds(s, N, K, bkt, false);
    for (int32_t i = 0; i < N; ++i) {
        int32_t j = SA[i] - 1;
        if (SA[i] > 0 && !stype[j]) SA[bkt[s[j]]++] = j;
    }
    bucket_bounds(s, N, K, bkt, true);
    for (int32_t i = N - 1; i >= 0; --i) {
        int32_t j = SA[i] - 1;
        if (SA[i] > 0 && stype[j]) SA[--bkt[s[j]]] = j;
    }
}

void sais(const int32_t *s, int32_t *SA, int32_t N, int32_t K) {
    std::vector<uint8_t> stype(N);
    stype[N - 1] = 1;
    for (int32_t i = N - 2; i >= 0; --i)
        stype[i] = (s[i] < s[i + 1] || (s[i] == s[i + 1] && stype[i + 1])) ? 1 : 0;
    auto lms = [&](int32_t i) { return i > 0 && stype[i] && !stype[i - 1]; };
    std::vector<int32_t> bkt(K);

    // 1. sort the LMS substrings: seed bucket ends with LMS positions, induce.
    bucket_bounds(s, N, K, bkt.data(), true);
    std::fill(SA, SA + N, -1);
    for (int32_t i = 1; i < N; ++i)
        if (lms(i)) SA[--bkt[s[i]]] = i;
    induce(s, SA, stype.data(), N, K, bkt.data());

    // 2. name the sorted LMS substrings.
    int32_t n1 = 0;
    for (int32_t i = 0; i < N; ++i)
        if (lms(SA[i])) SA[n1++] = SA[i];
    std::fill(SA + n1, SA + N, -1);
    int32_t name = 0, prev = -1;
    for (int32_t i = 0; i < n1; ++i) {
        int32_t pos = SA[i];
        bool diff = false;
        for (int32_t d = 0; d < N; ++d) {
            if (prev == -1 || s[pos + d] != s[prev + d] || stype[pos + d] != stype[prev + d]) {
                diff = true;
                break;
            }
            if (d > 0 && (lms(pos + d) || lms(prev + d))) break;
        }
        if (diff) {
            ++name;
            prev = pos;
        }
        SA[n1 + pos / 2] = name - 1;
    }
    for (int32_t i = N - 1, j = N - 1; i >= n1; --i)
        if (SA[i] >= 0) SA[j--] = SA[i];

    // 3. sort the reduced string (recursively if names repeat).
    int32_t *s1 = SA + N - n1;
    int32_t *SA1 = SA;
    if (name < n1) {
        std::vector<int32_t> s1copy(s1, s1 + n1);
        sais(s1copy.data(), SA1, n1, name);
    } else {
        for (int32_t i = 0; i < n1; ++i) SA1[s1[i]] = i;
    }

    // 4. induce the full order from the sorted LMS suffixes.
    bucket_bounds(s, N, K, bkt.data(), true);
    for (int32_t i = 1, j = 0; i < N; ++i)
        if (lms(i)) s1[j++] = i;
    for (int32_t i = 0; i < n1; ++i) SA1[i] = s1[SA1[i]];
    std::fill(SA + n1, SA + N, -1);
    for (int32_t i = n1 - 1; i >= 0; --i) {
        int32_t j = SA[i];
        SA[i] = -1;
        SA[--bkt[s[j]]] = j;
    }
    induce(s, SA, stype.data(), N, K, bkt.data());
}

}  // namespace

extern "C" ae_status ae_suffix_array(const uint8_t *codes, int64_t n, int32_t sigma, int32_t *sa) {
    if (n < 0 || sigma < 1 || sigma > 255 || (n > 0 && !codes) || !sa) return AE_EINVAL;
    if (n + 1 >= INT32_MAX) return AE_EUNSUPPORTED;
    int32_t N = (int32_t)n + 1;
    std::vector<int32_t> s;
    try {
        s.resize(N);
    } catch (...) {
        return AE_ENOMEM;
    }
    for (int64_t i = 0; i < n; ++i) {
        if (codes[i] >= sigma) return AE_EINVAL;
        s[i] = codes[i] + 1;
    }
    s[N - 1] = 0;
    if (N == 1) {
        sa[0] = 0;
        return AE_OK;
    }
    try {
        sais(s.data(), sa, N, sigma + 1);
    } catch (...) {
        return AE_ENOMEM;
    }
    return AE_OK;
}

// ------------------------------------------------------------------ index build

// The index of the text codes[0..n) from the suffix array `sa` (n + 1
// entries) of the reversed text followed by the sentinel (Section 5 (1)):
// position k < n of the reversed text holds T[n-1-k], so its suffix starting
// at k is the reverse of T[0..n-1-k], and the BWT letter of row h is the
// reversed text's letter before sa[h], T[n - sa[h]].
ae_status ae_host_index_fill(const uint8_t *codes, int64_t n, int32_t alphabet, const int32_t *sa, HostIndex *out) {
    memset(out, 0, sizeof(*out));
    int sigma = ae_alphabet_sigma(alphabet);
    if (!sigma || n < 1 || !sa) return AE_EINVAL;
    if (n + 1 >= INT32_MAX) return AE_EUNSUPPORTED;
    const int64_t N = n + 1;

    out->alphabet = alphabet;
    out->sigma = sigma;
    out->n = n;
    out->block_words = alphabet == AE_DNA ? AE_DNA_BLOCK_WORDS : AE_PROT_BLOCK_WORDS;
    out->nblocks = (N + AE_ROWS_PER_BLOCK - 1) / AE_ROWS_PER_BLOCK + 1;
    out->occ = (uint32_t *)calloc((size_t)(out->nblocks * out->block_words), sizeof(uint32_t));
    out->tend = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    out->text = (uint8_t *)malloc((size_t)n);
    if (!out->occ || !out->tend || !out->text) {
        ae_host_index_free(out);
        return AE_ENOMEM;
    }
    memcpy(out->text, codes, (size_t)n);

    // counts per letter for C[]
    std::vector<int64_t> cnt(sigma, 0);
    for (int64_t i = 0; i < n; ++i) ++cnt[codes[i]];
    out->C[0] = 1;
    for (int c = 0; c < sigma; ++c) out->C[c + 1] = out->C[c] + (uint32_t)cnt[c];

    std::vector<uint32_t> run(sigma, 0);
    out->dollar_row = -1;
    for (int64_t h = 0; h < N; ++h) {
        int64_t k = sa[h];
        if (k < 0 || k > n) {
            ae_host_index_free(out);
            return AE_EINVAL;
        }
        out->tend[h] = k < n ? (int32_t)(n - 1 - k) : -1;
        int code;
        if (k == 0) {
            out->dollar_row = h;
            code = 0;
        } else {
            code = codes[n - k];
        }
        int64_t b = h / AE_ROWS_PER_BLOCK, r = h % AE_ROWS_PER_BLOCK;
        uint32_t *blk = out->occ + b * out->block_words;
        if (r == 0)
            for (int c = 0; c < sigma; ++c) blk[c] = run[c];
        if (alphabet == AE_DNA) {
            blk[4 + r / 16] |= (uint32_t)code << (2 * (r % 16));
        } else {
            uint64_t *planes = (uint64_t *)(blk + 22);
            for (int t = 0; t < 5; ++t)
                if ((code >> t) & 1) planes[t] |= 1ull << r;
        }
        if (k != 0) ++run[code];
    }
    // trailing block(s): counts of everything, so a lookup at row N reads a valid block
    for (int64_t b = (N + AE_ROWS_PER_BLOCK - 1) / AE_ROWS_PER_BLOCK; b < out->nblocks; ++b) {
        uint32_t *blk = out->occ + b * out->block_words;
        for (int c = 0; c < sigma; ++c) blk[c] = run[c];
    }
    out->rows = N;
    return AE_OK;
}

// A collection (Section 2.3): the sequences are joined by a separator, code 0
// in the suffix array's alphabet (letters are code + 1), which sorts below every
// letter and never matches.  Row h of the BWT of the reversed joined text has
// suffix sa[h]; its BWT letter is the joined text's letter at J - sa[h] (J = the
// joined length).  Separator rows are counted in `sep`, not in the letter counts,
// and positions are mapped from the joined text to the sequences back to back.
ae_status ae_host_index_fill_collection(const uint8_t *codes, int64_t n, const int64_t *starts, int32_t nseq,
                                        int32_t alphabet, const int32_t *sa, HostIndex *out) {
    memset(out, 0, sizeof(*out));
    int sigma = ae_alphabet_sigma(alphabet);
    if (!sigma || n < 1 || !sa || nseq < 1 || !starts || starts[0] != 0) return AE_EINVAL;
    for (int32_t k = 1; k < nseq; ++k)
        if (starts[k] < starts[k - 1] || starts[k] > n) return AE_EINVAL;
    const int64_t nsep = nseq - 1, J = n + nsep, N = J + 1;
    if (N >= INT32_MAX) return AE_EUNSUPPORTED;
    out->alphabet = alphabet;
    out->sigma = sigma;
    out->n = n;
    out->rows = N;
    out->nseq = nseq;
    out->block_words = alphabet == AE_DNA ? AE_DNA_BLOCK_WORDS : AE_PROT_BLOCK_WORDS;
    out->nblocks = (N + AE_ROWS_PER_BLOCK - 1) / AE_ROWS_PER_BLOCK + 1;
    out->occ = (uint32_t *)calloc((size_t)(out->nblocks * out->block_words), sizeof(uint32_t));
    out->sep = (uint32_t *)calloc((size_t)(out->nblocks * AE_SEP_BLOCK_WORDS), sizeof(uint32_t));
    out->ends = (uint32_t *)calloc((size_t)((n + 31) / 32), sizeof(uint32_t));
    out->tend = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    out->text = (uint8_t *)malloc((size_t)n);
    std::vector<int64_t> jpos;   // joined position -> text position (-1 for a separator)
    std::vector<uint8_t> joined;
    try {
        jpos.resize((size_t)J);
        joined.resize((size_t)J);
    } catch (...) {
        ae_host_index_free(out);
        return AE_ENOMEM;
    }
    if (!out->occ || !out->sep || !out->ends || !out->tend || !out->text) {
        ae_host_index_free(out);
        return AE_ENOMEM;
    }
    memcpy(out->text, codes, (size_t)n);
    {
        int64_t q = 0;
        for (int32_t k = 0; k < nseq; ++k) {
            const int64_t b = starts[k], e = k + 1 < nseq ? starts[k + 1] : n;
            if (k > 0) {
                joined[q] = 0xFF;
                jpos[q++] = -1;
            }
            for (int64_t p = b; p < e; ++p) {
                joined[q] = codes[p];
                jpos[q++] = p;
            }
            if (e > b) out->ends[(e - 1) >> 5] |= 1u << ((e - 1) & 31);
        }
    }
    std::vector<int64_t> cnt(sigma, 0);
    for (int64_t i = 0; i < n; ++i) ++cnt[codes[i]];
    out->C[0] = (uint32_t)(1 + nsep);
    for (int c = 0; c < sigma; ++c) out->C[c + 1] = out->C[c] + (uint32_t)cnt[c];

    std::vector<uint32_t> run(sigma, 0);
    uint32_t seps = 0;
    out->dollar_row = -1;
    for (int64_t h = 0; h < N; ++h) {
        const int64_t k = sa[h];
        if (k < 0 || k > J) {
            ae_host_index_free(out);
            return AE_EINVAL;
        }
        // the substrings of row h end at joined position J - 1 - k
        out->tend[h] = (k < J && jpos[J - 1 - k] >= 0) ? (int32_t)jpos[J - 1 - k] : -1;
        int code = 0;
        bool is_sep = false;
        if (k == 0) {
            out->dollar_row = h;
        } else if (joined[J - k] == 0xFF) {
            is_sep = true;
        } else {
            code = joined[J - k];
        }
        const int64_t b = h / AE_ROWS_PER_BLOCK, r = h % AE_ROWS_PER_BLOCK;
        uint32_t *blk = out->occ + b * out->block_words;
        uint32_t *sb = out->sep + b * AE_SEP_BLOCK_WORDS;
        if (r == 0) {
            for (int c = 0; c < sigma; ++c) blk[c] = run[c];
            sb[0] = seps;
        }
        if (alphabet == AE_DNA) {
            blk[4 + r / 16] |= (uint32_t)code << (2 * (r % 16));
        } else {
            uint64_t *planes = (uint64_t *)(blk + 22);
            for (int t = 0; t < 5; ++t)
                if ((code >> t) & 1) planes[t] |= 1ull << r;
        }
        if (is_sep) {
            sb[1 + r / 32] |= 1u << (r % 32);
            ++seps;
        } else if (k != 0) {
            ++run[code];
        }
    }
    for (int64_t b = (N + AE_ROWS_PER_BLOCK - 1) / AE_ROWS_PER_BLOCK; b < out->nblocks; ++b) {
        uint32_t *blk = out->occ + b * out->block_words;
        for (int c = 0; c < sigma; ++c) blk[c] = run[c];
        out->sep[b * AE_SEP_BLOCK_WORDS] = seps;
    }
    return AE_OK;
}

void ae_host_index_free(HostIndex *h) {
    if (!h) return;
    free(h->occ);
    free(h->tend);
    free(h->text);
    free(h->sep);
    free(h->ends);
    h->occ = nullptr;
    h->tend = nullptr;
    h->text = nullptr;
    h->sep = nullptr;
    h->ends = nullptr;
}

// ------------------------------------------------------------------ file format
// header: magic "AEIDX\0v1", then int64 fields, then the three arrays, then an
// FNV-1a 64-bit checksum of everything before it.

namespace {
const char kMagic[8] = {'A', 'E', 'I', 'D', 'X', 0, 'v', '1'};

struct Fnv {
    uint64_t h = 1469598103934665603ull;
    void add(const void *p, size_t n) {
        const uint8_t *b = (const uint8_t *)p;
        for (size_t i = 0; i < n; ++i) {
            h ^= b[i];
            h *= 1099511628211ull;
        }
    }
};

bool wr(FILE *f, Fnv &fnv, const void *p, size_t n) {
    fnv.add(p, n);
    return fwrite(p, 1, n, f) == n;
}
bool rd(FILE *f, Fnv &fnv, void *p, size_t n) {
    if (fread(p, 1, n, f) != n) return false;
    fnv.add(p, n);
    return true;
}
}  // namespace

ae_status ae_host_index_save(const HostIndex *h, const char *path) {
    FILE *f = fopen(path, "wb");
    if (!f) return AE_EIO;
    Fnv fnv;
    // header words 6 and 7: sequences and BWT rows of a collection (0, 0 for one text)
    int64_t hdr[8] = {h->alphabet, h->sigma, h->n, h->dollar_row, h->nblocks, h->block_words,
                      h->nseq, h->nseq ? h->rows : 0};
    bool ok = wr(f, fnv, kMagic, 8) && wr(f, fnv, hdr, sizeof(hdr)) && wr(f, fnv, h->C, sizeof(h->C)) &&
              wr(f, fnv, h->occ, sizeof(uint32_t) * (size_t)(h->nblocks * h->block_words)) &&
              wr(f, fnv, h->tend, sizeof(int32_t) * (size_t)h->rows) && wr(f, fnv, h->text, (size_t)h->n);
    if (h->nseq)
        ok = ok && wr(f, fnv, h->sep, sizeof(uint32_t) * (size_t)(h->nblocks * AE_SEP_BLOCK_WORDS)) &&
             wr(f, fnv, h->ends, sizeof(uint32_t) * (size_t)((h->n + 31) / 32));
    uint64_t sum = fnv.h;
    ok = ok && fwrite(&sum, 1, 8, f) == 8;
    ok = (fclose(f) == 0) && ok;
    return ok ? AE_OK : AE_EIO;
}

ae_status ae_host_index_load(const char *path, HostIndex *h) {
    memset(h, 0, sizeof(*h));
    FILE *f = fopen(path, "rb");
    if (!f) return AE_EIO;
    Fnv fnv;
    char magic[8];
    int64_t hdr[8];
    ae_status st = AE_EIO;
    if (!rd(f, fnv, magic, 8) || memcmp(magic, kMagic, 8) != 0 || !rd(f, fnv, hdr, sizeof(hdr))) goto done;
    h->alphabet = (int32_t)hdr[0];
    h->sigma = (int32_t)hdr[1];
    h->n = hdr[2];
    h->dollar_row = hdr[3];
    h->nblocks = hdr[4];
    h->block_words = (int32_t)hdr[5];
    h->nseq = (int32_t)hdr[6];
    h->rows = h->nseq ? hdr[7] : h->n + 1;
    if (ae_alphabet_sigma(h->alphabet) != h->sigma || h->n < 1 || h->rows >= INT32_MAX || h->nseq < 0 ||
        h->rows != h->n + (h->nseq ? h->nseq : 1) ||
        h->nblocks != (h->rows + AE_ROWS_PER_BLOCK - 1) / AE_ROWS_PER_BLOCK + 1 ||
        h->block_words != (h->alphabet == AE_DNA ? AE_DNA_BLOCK_WORDS : AE_PROT_BLOCK_WORDS))
        goto done;
    if (!rd(f, fnv, h->C, sizeof(h->C))) goto done;
    h->occ = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(h->nblocks * h->block_words));
    h->tend = (int32_t *)malloc(sizeof(int32_t) * (size_t)h->rows);
    h->text = (uint8_t *)malloc((size_t)h->n);
    if (h->nseq) {
        h->sep = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(h->nblocks * AE_SEP_BLOCK_WORDS));
        h->ends = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)((h->n + 31) / 32));
    }
    if (!h->occ || !h->tend || !h->text || (h->nseq && (!h->sep || !h->ends))) {
        st = AE_ENOMEM;
        goto done;
    }
    if (!rd(f, fnv, h->occ, sizeof(uint32_t) * (size_t)(h->nblocks * h->block_words)) ||
        !rd(f, fnv, h->tend, sizeof(int32_t) * (size_t)h->rows) || !rd(f, fnv, h->text, (size_t)h->n))
        goto done;
    if (h->nseq && (!rd(f, fnv, h->sep, sizeof(uint32_t) * (size_t)(h->nblocks * AE_SEP_BLOCK_WORDS)) ||
                    !rd(f, fnv, h->ends, sizeof(uint32_t) * (size_t)((h->n + 31) / 32))))
        goto done;
    {
        uint64_t want = fnv.h, got = 0;
        if (fread(&got, 1, 8, f) != 8 || got != want) goto done;
    }
    st = AE_OK;
done:
    fclose(f);
    if (st != AE_OK) ae_host_index_free(h);
    return st;
}
