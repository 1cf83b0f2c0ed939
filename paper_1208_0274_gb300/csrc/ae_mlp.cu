// Search-work predictor: query features, a 66-128-128-2 perceptron with its
// forward and backward passes on the bf16 tensor cores, and Adam training.
// The C ABI is declared in include/ae_mlp.h.  Nothing here changes a search
// result; the engine only reads the predictions as buffer-size hints.

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "ae_device.cuh"
#include "ae_internal.h"
#include "ae_kernels.h"
#include "ae_mlp.h"

namespace {

constexpr int NIN = AE_MLP_IN, NH = AE_MLP_HIDDEN, NOUT = AE_MLP_OUT;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NH * NIN, OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH,
              OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NOUT * NH, NPARAM = OFF_B3 + NOUT;
static_assert(NPARAM == AE_MLP_PARAMS, "packed parameter count");

// norm buffer: x_mu[66] | x_isd[66] | y_mu[2] | y_sd[2]
constexpr int NORM_XMU = 0, NORM_XISD = NIN, NORM_YMU = 2 * NIN, NORM_YSD = 2 * NIN + NOUT,
              NORM_SIZE = 2 * NIN + 2 * NOUT;

// ------------------------------------------------------------------ tensor-core GEMM
//
// C(m, n) = sum_k A(m, k) B(k, n) with A(m, k) = A[m*sam + k*sak] and
// B(k, n) = B[k*sbk + n*sbn] (fp32 in memory, rounded to bf16 for the
// product, fp32 accumulate).  Epilogue per element: + bias[n]; Z = that value
// (pre-activation); zeroed where mask <= 0; relu; stored to C (ld ldc).  One
// warp owns a 16 x 32 tile (four m16n8k16 products per k step of 16).
//
// Split K: the weight gradients are products with a small output (at most
// 128 x 128) and K = the batch rows, which a few warps would walk alone.  With
// `part` set, gemm() splits K into up to GEMM_KSPLIT_MAX chunks (blockIdx.y),
// each block stores its raw partial tile to part[s][M][N], and k_gemm_reduce
// sums the chunks in chunk order and applies the epilogue, so the result does
// not depend on scheduling.

struct GemmArgs {
    const float *A;
    int64_t sam, sak;
    const float *B;
    int64_t sbk, sbn;
    float *C;
    int64_t ldc;
    const float *bias;
    const float *mask;
    float *Z;
    int M, N, K, relu;
    float *part;        // split-K partials (GEMM_KSPLIT_MAX * M * N floats), or null
    int kchunk;         // K per chunk (a multiple of 16); set by gemm()
};

constexpr int GEMM_NT = 4;      // n8 sub-tiles per warp
constexpr int GEMM_WARPS = 4;
constexpr int GEMM_KSPLIT_MAX = 64;
constexpr int GEMM_TARGET_BLOCKS = 2 * 152;

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);   // .x (low half) = lo
    return *reinterpret_cast<uint32_t *>(&v);
}

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__global__ void __launch_bounds__(GEMM_WARPS * 32) k_gemm(GemmArgs a) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int64_t tiles_n = (a.N + 8 * GEMM_NT - 1) / (8 * GEMM_NT);
    const int64_t tiles_m = (a.M + 15) / 16;
    const int64_t tile = (int64_t)blockIdx.x * GEMM_WARPS + warp;
    if (tile >= tiles_m * tiles_n) return;
    const int m0 = (int)(tile / tiles_n) * 16, n0 = (int)(tile % tiles_n) * 8 * GEMM_NT;
    const int kbeg = (int)blockIdx.y * a.kchunk, kend = min(a.K, kbeg + a.kchunk);
    auto ldA = [&](int m, int k) -> float {
        return (m < a.M && k < kend) ? a.A[(int64_t)m * a.sam + (int64_t)k * a.sak] : 0.f;
    };
    auto ldB = [&](int k, int n) -> float {
        return (k < kend && n < a.N) ? a.B[(int64_t)k * a.sbk + (int64_t)n * a.sbn] : 0.f;
    };
    float acc[GEMM_NT][4];
#pragma unroll
    for (int j = 0; j < GEMM_NT; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
    for (int k0 = kbeg; k0 < kend; k0 += 16) {
        // A fragment (16 x 16, row major): rows g and g+8, columns 2t, 2t+1 and 2t+8, 2t+9
        uint32_t ra[4];
        ra[0] = pack_bf16x2(ldA(m0 + g, k0 + 2 * t), ldA(m0 + g, k0 + 2 * t + 1));
        ra[1] = pack_bf16x2(ldA(m0 + g + 8, k0 + 2 * t), ldA(m0 + g + 8, k0 + 2 * t + 1));
        ra[2] = pack_bf16x2(ldA(m0 + g, k0 + 2 * t + 8), ldA(m0 + g, k0 + 2 * t + 9));
        ra[3] = pack_bf16x2(ldA(m0 + g + 8, k0 + 2 * t + 8), ldA(m0 + g + 8, k0 + 2 * t + 9));
#pragma unroll
        for (int j = 0; j < GEMM_NT; ++j) {
            // B fragment (16 x 8, column major): rows 2t, 2t+1 and 2t+8, 2t+9 of column g
            const int n = n0 + 8 * j + g;
            const uint32_t b0 = pack_bf16x2(ldB(k0 + 2 * t, n), ldB(k0 + 2 * t + 1, n));
            const uint32_t b1 = pack_bf16x2(ldB(k0 + 2 * t + 8, n), ldB(k0 + 2 * t + 9, n));
            mma_bf16_16816(acc[j], ra, b0, b1);
        }
    }
#pragma unroll
    for (int j = 0; j < GEMM_NT; ++j) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            // accumulator layout: rows g (i < 2) and g+8 (i >= 2), columns 2t + (i & 1)
            const int row = m0 + g + (i >= 2 ? 8 : 0);
            const int col = n0 + 8 * j + 2 * t + (i & 1);
            if (row >= a.M || col >= a.N) continue;
            if (gridDim.y > 1) {
                a.part[((int64_t)blockIdx.y * a.M + row) * a.N + col] = acc[j][i];
                continue;
            }
            float v = acc[j][i] + (a.bias ? a.bias[col] : 0.f);
            const int64_t idx = (int64_t)row * a.ldc + col;
            if (a.Z) a.Z[idx] = v;
            if (a.mask && !(a.mask[idx] > 0.f)) v = 0.f;
            if (a.relu) v = fmaxf(v, 0.f);
            a.C[idx] = v;
        }
    }
}

int grid1(int64_t n, int threads) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + threads - 1) / threads, 4096));
}

// sum of the split-K partials in chunk order, then the epilogue of k_gemm
__global__ void k_gemm_reduce(GemmArgs a, int nsplit) {
    const int64_t total = (int64_t)a.M * a.N;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int row = (int)(e / a.N), col = (int)(e % a.N);
        float v = 0.f;
        for (int s = 0; s < nsplit; ++s) v += a.part[(int64_t)s * total + e];
        v += a.bias ? a.bias[col] : 0.f;
        const int64_t idx = (int64_t)row * a.ldc + col;
        if (a.Z) a.Z[idx] = v;
        if (a.mask && !(a.mask[idx] > 0.f)) v = 0.f;
        if (a.relu) v = fmaxf(v, 0.f);
        a.C[idx] = v;
    }
}

void gemm(GemmArgs a, cudaStream_t st) {
    if (a.M <= 0 || a.N <= 0) return;
    const int64_t tiles = ((a.M + 15) / 16) * ((a.N + 8 * GEMM_NT - 1) / (8 * GEMM_NT));
    const int64_t blocks = (tiles + GEMM_WARPS - 1) / GEMM_WARPS;
    const int ksteps = (a.K + 15) / 16;
    // chunks of at least 4 k steps, enough of them to fill the GPU
    int nsplit = 1;
    if (a.part && blocks < GEMM_TARGET_BLOCKS && ksteps >= 8)
        nsplit = (int)std::min<int64_t>({GEMM_KSPLIT_MAX, (GEMM_TARGET_BLOCKS + blocks - 1) / blocks, ksteps / 4});
    const int steps_per = (ksteps + nsplit - 1) / nsplit;
    a.kchunk = 16 * std::max(steps_per, 1);
    nsplit = std::max(1, (a.K + a.kchunk - 1) / a.kchunk);
    ++g_launches;
    k_gemm<<<dim3((unsigned)blocks, (unsigned)nsplit), GEMM_WARPS * 32, 0, st>>>(a);
    if (nsplit > 1) {
        ++g_launches;
        k_gemm_reduce<<<grid1((int64_t)a.M * a.N, 256), 256, 0, st>>>(a, nsplit);
    }
}

// ------------------------------------------------------------------ elementwise kernels

__global__ void k_standardize(const float *x, const float *norm, float *out, int64_t rows) {
    const int64_t total = rows * NIN;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % NIN);
        out[i] = (x[i] - norm[NORM_XMU + c]) * norm[NORM_XISD + c];
    }
}

__global__ void k_denorm(const float *y, const float *norm, float *out, int64_t rows) {
    const int64_t total = rows * NOUT;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % NOUT);
        out[i] = y[i] * norm[NORM_YSD + c] + norm[NORM_YMU + c];
    }
}

// Residuals against the normalised targets, dL/dy = r / B, and L = sum r^2 / (2B)
// written to *loss (one block; fixed summation order).
__global__ void k_loss(const float *y, const float *t, const float *norm, float *dy, int rows, float *loss) {
    __shared__ float part[256];
    float s = 0.f;
    const float inv_b = 1.f / (float)rows;
    for (int i = threadIdx.x; i < rows * NOUT; i += blockDim.x) {
        const int c = i % NOUT;
        const float tn = (t[i] - norm[NORM_YMU + c]) / norm[NORM_YSD + c];
        const float r = y[i] - tn;
        dy[i] = r * inv_b;
        s += r * r;
    }
    part[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = part[0] * 0.5f * inv_b;
}

// out[c] = sum over rows of src[r*N + c]; one warp per column.
__global__ void k_colsum(const float *src, int rows, int N, float *out) {
    const int lane = threadIdx.x & 31;
    const int col = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (col >= N) return;
    float s = 0.f;
    for (int r = lane; r < rows; r += 32) s += src[(int64_t)r * N + col];
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
    if (lane == 0) out[col] = s;
}

// Adam (Kingma and Ba, 2015) with decoupled weight decay (Loshchilov and
// Hutter, 2019): p -= lr * (m_hat / (sqrt(v_hat) + eps) + wd * p).
__global__ void k_adam(float *p, const float *g, float *m, float *v, int n, float lr, float bc1, float bc2, float wd) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float pi = p[i];
        p[i] = pi - lr * ((mi / bc1) / (sqrtf(vi / bc2) + eps) + wd * pi);
    }
}

__global__ void k_gather(const float *x, const float *t, const int32_t *perm, int rows, float *xb, float *tb) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < rows * NIN; i += gridDim.x * blockDim.x) {
        const int r = i / NIN, c = i % NIN;
        xb[i] = x[(int64_t)perm[r] * NIN + c];
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < rows * NOUT; i += gridDim.x * blockDim.x) {
        const int r = i / NOUT, c = i % NOUT;
        tb[i] = t[(int64_t)perm[r] * NOUT + c];
    }
}

// ------------------------------------------------------------------ features

// Window length of the interval feature: ceil(log4(n + 1)) + 4 letters, long
// enough that a window of an unrelated query is rarely found in the text.
int interval_window(int64_t n) {
    int k = 0;
    for (int64_t r = 1; r < n + 1; r *= 4) ++k;
    return std::min(k + 4, 32);
}

__device__ __forceinline__ int dna_code(uint8_t ch, int *bad) {
    switch (ch) {
        case 'A': return 0;
        case 'C': return 1;
        case 'G': return 2;
        case 'T': return 3;
        default: atomicExch(bad, 1); return 0;
    }
}

// One block per query: the 3-mer spectrum, log1p(m), and the mean over the
// query's windows of K letters of log1p(|SA interval of the window|).  The
// interval of a window w comes from K backward steps with w's letters in
// order, which give the rows of reverse(w) in the index of the reversed text,
// one row per occurrence of w in T (Section 2.3, Section 5 (3)).
constexpr int FEAT_THREADS = 128;

__global__ void __launch_bounds__(FEAT_THREADS) k_features(IndexView ix, const uint8_t *seq, const int64_t *off,
                                                           int nq, int K, float *feat, int *bad) {
    __shared__ int cnt[64];
    __shared__ float part[FEAT_THREADS];
    const int q = blockIdx.x;
    if (q >= nq) return;
    for (int w = threadIdx.x; w < 64; w += blockDim.x) cnt[w] = 0;
    __syncthreads();
    const int64_t b = off[q], m = off[q + 1] - off[q];
    for (int64_t p = threadIdx.x; p < m; p += blockDim.x) {
        const int c0 = dna_code(seq[b + p], bad);
        if (p + 2 < m) atomicAdd(&cnt[16 * c0 + 4 * dna_code(seq[b + p + 1], bad) + dna_code(seq[b + p + 2], bad)], 1);
    }
    float acc = 0.f;
    for (int64_t p = threadIdx.x; p + K <= m; p += blockDim.x) {
        uint32_t lo = 0, hi = (uint32_t)ix.rows;
        for (int s = 0; s < K && lo < hi; ++s) {
            const int c = dna_code(seq[b + p + s], bad);
            lo = ix.C[c] + aedev::occ_dna(ix, c, lo);
            hi = ix.C[c] + aedev::occ_dna(ix, c, hi);
        }
        acc += log1pf(lo < hi ? (float)(hi - lo) : 0.f);
    }
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int w = FEAT_THREADS / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    const float inv = m >= 3 ? 1.f / (float)(m - 2) : 0.f;
    for (int w = threadIdx.x; w < 64; w += blockDim.x) feat[(int64_t)q * NIN + w] = (float)cnt[w] * inv;
    if (threadIdx.x == 0) {
        feat[(int64_t)q * NIN + 64] = log1pf((float)m);
        feat[(int64_t)q * NIN + 65] = m >= K ? part[0] / (float)(m - K + 1) : 0.f;
    }
}

uint64_t splitmix64(uint64_t &s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Per-thread device scratch of ae_mlp_features (offsets and error
// flag), grown on demand and kept so that calls allocate nothing once warm.
struct FeatScratch {
    int64_t *off = nullptr;
    int *bad = nullptr;
    int *h_bad = nullptr;
    int32_t cap = 0;
    void release() {
        if (off) cudaFree(off);
        if (bad) cudaFree(bad);
        if (h_bad) cudaFreeHost(h_bad);
        off = nullptr, bad = nullptr, h_bad = nullptr;
        cap = 0;
    }
    ~FeatScratch() { release(); }
};
thread_local FeatScratch g_feat_scratch;

struct mlp_error {
    ae_status st;
};

#define MC(x)                                                          \
    do {                                                               \
        if ((x) != cudaSuccess) throw mlp_error{AE_ECUDA};             \
    } while (0)

}  // namespace

struct ae_mlp {
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr, *norm = nullptr;
    int64_t step = 0;
    int32_t cap = 0;
    float *x = nullptr, *z1 = nullptr, *a1 = nullptr, *z2 = nullptr, *a2 = nullptr, *y = nullptr, *dy = nullptr,
          *d1 = nullptr, *d2 = nullptr, *xb = nullptr, *tb = nullptr, *loss = nullptr;
    float *part = nullptr;          // split-K partials of the weight gradients
    int32_t *perm = nullptr;
    int32_t perm_cap = 0, loss_cap = 0;
    float h_norm[NORM_SIZE];

    void free_acts() {
        float **bufs[] = {&x, &z1, &a1, &z2, &a2, &y, &dy, &d1, &d2, &xb, &tb};
        for (float **b : bufs) {
            if (*b) cudaFree(*b);
            *b = nullptr;
        }
        cap = 0;
    }
    ~ae_mlp() {
        free_acts();
        for (float *b : {p, g, m, v, norm, loss, part})
            if (b) cudaFree(b);
        if (perm) cudaFree(perm);
    }
    void reserve(int32_t rows) {
        if (rows <= cap) return;
        free_acts();
        const int32_t c = std::max(rows, 256);
        const size_t in = sizeof(float) * (size_t)c * NIN, hid = sizeof(float) * (size_t)c * NH,
                     out = sizeof(float) * (size_t)c * NOUT;
        struct {
            float **b;
            size_t bytes;
        } plan[] = {{&x, in}, {&z1, hid}, {&a1, hid}, {&z2, hid}, {&a2, hid}, {&y, out},
                    {&dy, out}, {&d1, hid}, {&d2, hid}, {&xb, in}, {&tb, out}};
        for (auto &e : plan)
            if (cudaMalloc(e.b, e.bytes) != cudaSuccess) {
                cudaGetLastError();
                free_acts();
                throw mlp_error{AE_ENOMEM};
            }
        cap = c;
    }

    // forward of `rows` standardised inputs already in x
    void forward_std(int32_t rows, cudaStream_t st) {
        GemmArgs a{};
        a.A = x, a.sam = NIN, a.sak = 1, a.B = p + OFF_W1, a.sbk = 1, a.sbn = NIN, a.C = a1, a.ldc = NH;
        a.bias = p + OFF_B1, a.Z = z1, a.M = rows, a.N = NH, a.K = NIN, a.relu = 1;
        gemm(a, st);
        a = GemmArgs{};
        a.A = a1, a.sam = NH, a.sak = 1, a.B = p + OFF_W2, a.sbk = 1, a.sbn = NH, a.C = a2, a.ldc = NH;
        a.bias = p + OFF_B2, a.Z = z2, a.M = rows, a.N = NH, a.K = NH, a.relu = 1;
        gemm(a, st);
        a = GemmArgs{};
        a.A = a2, a.sam = NH, a.sak = 1, a.B = p + OFF_W3, a.sbk = 1, a.sbn = NH, a.C = y, a.ldc = NOUT;
        a.bias = p + OFF_B3, a.M = rows, a.N = NOUT, a.K = NH;
        gemm(a, st);
    }

    // loss and gradients (into g) of `rows` inputs in x with raw targets t
    void backward(int32_t rows, const float *t, float *loss_slot, cudaStream_t st) {
        forward_std(rows, st);
        ++g_launches;
        k_loss<<<1, 256, 0, st>>>(y, t, norm, dy, rows, loss_slot);
        GemmArgs a{};
        // dW3 = dy^T a2
        a.A = dy, a.sam = 1, a.sak = NOUT, a.B = a2, a.sbk = NH, a.sbn = 1, a.C = g + OFF_W3, a.ldc = NH;
        a.M = NOUT, a.N = NH, a.K = rows;
        a.part = part;
        gemm(a, st);
        colsum(dy, rows, NOUT, g + OFF_B3, st);
        // d2 = (dy W3) * [z2 > 0]
        a = GemmArgs{};
        a.A = dy, a.sam = NOUT, a.sak = 1, a.B = p + OFF_W3, a.sbk = NH, a.sbn = 1, a.C = d2, a.ldc = NH;
        a.mask = z2, a.M = rows, a.N = NH, a.K = NOUT;
        gemm(a, st);
        // dW2 = d2^T a1
        a = GemmArgs{};
        a.A = d2, a.sam = 1, a.sak = NH, a.B = a1, a.sbk = NH, a.sbn = 1, a.C = g + OFF_W2, a.ldc = NH;
        a.M = NH, a.N = NH, a.K = rows;
        a.part = part;
        gemm(a, st);
        colsum(d2, rows, NH, g + OFF_B2, st);
        // d1 = (d2 W2) * [z1 > 0]
        a = GemmArgs{};
        a.A = d2, a.sam = NH, a.sak = 1, a.B = p + OFF_W2, a.sbk = NH, a.sbn = 1, a.C = d1, a.ldc = NH;
        a.mask = z1, a.M = rows, a.N = NH, a.K = NH;
        gemm(a, st);
        // dW1 = d1^T x
        a = GemmArgs{};
        a.A = d1, a.sam = 1, a.sak = NH, a.B = x, a.sbk = NIN, a.sbn = 1, a.C = g + OFF_W1, a.ldc = NIN;
        a.M = NH, a.N = NIN, a.K = rows;
        a.part = part;
        gemm(a, st);
        colsum(d1, rows, NH, g + OFF_B1, st);
    }

    static void colsum(const float *src, int rows, int N, float *out, cudaStream_t st) {
        ++g_launches;
        k_colsum<<<(N + 3) / 4, 128, 0, st>>>(src, rows, N, out);
    }

    void standardize(const float *raw, int32_t rows, float *dst, cudaStream_t st) {
        ++g_launches;
        k_standardize<<<grid1((int64_t)rows * NIN, 256), 256, 0, st>>>(raw, norm, dst, rows);
    }

    void adam_step(float lr, float wd, cudaStream_t st) {
        ++step;
        const double bc1 = 1.0 - std::pow(0.9, (double)step), bc2 = 1.0 - std::pow(0.999, (double)step);
        ++g_launches;
        k_adam<<<grid1(NPARAM, 256), 256, 0, st>>>(p, g, m, v, NPARAM, lr, (float)bc1, (float)bc2, wd);
    }
};

extern "C" {

ae_status ae_mlp_create(uint64_t seed, ae_mlp **out) {
    if (!out) return AE_EINVAL;
    *out = nullptr;
    ae_mlp *mlp = new (std::nothrow) ae_mlp();
    if (!mlp) return AE_ENOMEM;
    try {
        for (float **b : {&mlp->p, &mlp->g, &mlp->m, &mlp->v})
            if (cudaMalloc(b, sizeof(float) * NPARAM) != cudaSuccess) throw mlp_error{AE_ENOMEM};
        if (cudaMalloc(&mlp->norm, sizeof(float) * NORM_SIZE) != cudaSuccess) throw mlp_error{AE_ENOMEM};
        if (cudaMalloc(&mlp->part, sizeof(float) * GEMM_KSPLIT_MAX * NH * NH) != cudaSuccess)
            throw mlp_error{AE_ENOMEM};
        std::vector<float> h(NPARAM, 0.f);
        uint64_t s = seed;
        auto fill = [&](int off, int rows, int cols) {
            const double bound = std::sqrt(6.0 / cols);
            for (int i = 0; i < rows * cols; ++i) {
                const double u = (double)(splitmix64(s) >> 11) * (1.0 / 9007199254740992.0);
                h[off + i] = (float)((2.0 * u - 1.0) * bound);
            }
        };
        fill(OFF_W1, NH, NIN);
        fill(OFF_W2, NH, NH);
        fill(OFF_W3, NOUT, NH);
        MC(cudaMemcpy(mlp->p, h.data(), sizeof(float) * NPARAM, cudaMemcpyHostToDevice));
        MC(cudaMemset(mlp->m, 0, sizeof(float) * NPARAM));
        MC(cudaMemset(mlp->v, 0, sizeof(float) * NPARAM));
        MC(cudaMemset(mlp->g, 0, sizeof(float) * NPARAM));
        for (int i = 0; i < NIN; ++i) {
            mlp->h_norm[NORM_XMU + i] = 0.f;
            mlp->h_norm[NORM_XISD + i] = 1.f;
        }
        for (int i = 0; i < NOUT; ++i) {
            mlp->h_norm[NORM_YMU + i] = 0.f;
            mlp->h_norm[NORM_YSD + i] = 1.f;
        }
        MC(cudaMemcpy(mlp->norm, mlp->h_norm, sizeof(float) * NORM_SIZE, cudaMemcpyHostToDevice));
    } catch (const mlp_error &e) {
        cudaGetLastError();
        delete mlp;
        return e.st;
    }
    *out = mlp;
    return AE_OK;
}

void ae_mlp_free(ae_mlp *mlp) { delete mlp; }

ae_status ae_mlp_set_params(ae_mlp *mlp, const float *params) {
    if (!mlp || !params) return AE_EINVAL;
    if (cudaMemcpy(mlp->p, params, sizeof(float) * NPARAM, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(mlp->m, 0, sizeof(float) * NPARAM) != cudaSuccess ||
        cudaMemset(mlp->v, 0, sizeof(float) * NPARAM) != cudaSuccess)
        return AE_ECUDA;
    mlp->step = 0;
    return AE_OK;
}

ae_status ae_mlp_get_params(const ae_mlp *mlp, float *params) {
    if (!mlp || !params) return AE_EINVAL;
    return cudaMemcpy(params, mlp->p, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost) == cudaSuccess ? AE_OK
                                                                                                       : AE_ECUDA;
}

ae_status ae_mlp_set_norm(ae_mlp *mlp, const float *x_mu, const float *x_sd, const float *y_mu, const float *y_sd) {
    if (!mlp || !x_mu || !x_sd || !y_mu || !y_sd) return AE_EINVAL;
    for (int i = 0; i < NIN; ++i)
        if (!(x_sd[i] > 0.f)) return AE_EINVAL;
    for (int i = 0; i < NOUT; ++i)
        if (!(y_sd[i] > 0.f)) return AE_EINVAL;
    for (int i = 0; i < NIN; ++i) {
        mlp->h_norm[NORM_XMU + i] = x_mu[i];
        mlp->h_norm[NORM_XISD + i] = 1.f / x_sd[i];
    }
    for (int i = 0; i < NOUT; ++i) {
        mlp->h_norm[NORM_YMU + i] = y_mu[i];
        mlp->h_norm[NORM_YSD + i] = y_sd[i];
    }
    return cudaMemcpy(mlp->norm, mlp->h_norm, sizeof(float) * NORM_SIZE, cudaMemcpyHostToDevice) == cudaSuccess
               ? AE_OK
               : AE_ECUDA;
}

ae_status ae_mlp_features(const ae_index *idx, const uint8_t *d_seq, const int64_t *offsets, int32_t nq,
                          float *d_feat, void *stream) {
    if (!idx || !offsets || nq < 0 || (nq > 0 && !d_feat)) return AE_EINVAL;
    if (nq == 0) return AE_OK;
    if (offsets[0] != 0) return AE_EINVAL;
    for (int q = 0; q < nq; ++q)
        if (offsets[q + 1] < offsets[q]) return AE_EINVAL;
    if (offsets[nq] > 0 && !d_seq) return AE_EINVAL;
    const IndexView *ix = ae_index_view(idx);
    if (ix->alphabet != AE_DNA) return AE_EUNSUPPORTED;
    cudaStream_t st = (cudaStream_t)stream;
    FeatScratch &fs = g_feat_scratch;
    if (fs.cap < nq + 1) {
        fs.release();
        const int32_t c = std::max(nq + 1, 1024);
        if (cudaMalloc(&fs.off, sizeof(int64_t) * c) != cudaSuccess || cudaMalloc(&fs.bad, sizeof(int)) != cudaSuccess ||
            cudaMallocHost(&fs.h_bad, sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            fs.release();
            return AE_ENOMEM;
        }
        fs.cap = c;
    }
    if (cudaMemcpyAsync(fs.off, offsets, sizeof(int64_t) * (nq + 1), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(fs.bad, 0, sizeof(int), st) != cudaSuccess)
        return AE_ECUDA;
    ++g_launches;
    k_features<<<nq, FEAT_THREADS, 0, st>>>(*ix, d_seq, fs.off, nq, interval_window(ix->n), d_feat, fs.bad);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(fs.h_bad, fs.bad, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return AE_ECUDA;
    return *fs.h_bad ? AE_EINVAL : AE_OK;
}

ae_status ae_mlp_forward(ae_mlp *mlp, const float *d_x, int32_t B, float *d_y, void *stream) {
    if (!mlp || B < 0 || (B > 0 && (!d_x || !d_y))) return AE_EINVAL;
    if (B == 0) return AE_OK;
    cudaStream_t st = (cudaStream_t)stream;
    try {
        mlp->reserve(B);
        mlp->standardize(d_x, B, mlp->x, st);
        mlp->forward_std(B, st);
        ++g_launches;
        k_denorm<<<grid1((int64_t)B * NOUT, 256), 256, 0, st>>>(mlp->y, mlp->norm, d_y, B);
        MC(cudaGetLastError());
        MC(cudaStreamSynchronize(st));
    } catch (const mlp_error &e) {
        cudaGetLastError();
        return e.st;
    }
    return AE_OK;
}

ae_status ae_mlp_loss_grad(ae_mlp *mlp, const float *d_x, const float *d_t, int32_t B, float *loss, float *grads,
                           void *stream) {
    if (!mlp || B < 1 || !d_x || !d_t || !loss) return AE_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    try {
        mlp->reserve(B);
        if (mlp->loss_cap < 1) {
            MC(cudaMalloc(&mlp->loss, sizeof(float) * 1024));
            mlp->loss_cap = 1024;
        }
        mlp->standardize(d_x, B, mlp->x, st);
        mlp->backward(B, d_t, mlp->loss, st);
        MC(cudaGetLastError());
        MC(cudaMemcpyAsync(loss, mlp->loss, sizeof(float), cudaMemcpyDeviceToHost, st));
        if (grads) MC(cudaMemcpyAsync(grads, mlp->g, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost, st));
        MC(cudaStreamSynchronize(st));
    } catch (const mlp_error &e) {
        cudaGetLastError();
        return e.st;
    }
    return AE_OK;
}

ae_status ae_mlp_train(ae_mlp *mlp, const float *d_x, const float *d_t, int32_t n, int32_t epochs, int32_t batch,
                       float lr, float weight_decay, uint64_t seed, float *loss, void *stream) {
    if (!mlp || n < 1 || !d_x || !d_t || epochs < 0 || batch < 1 || !(lr > 0.f) || !(weight_decay >= 0.f))
        return AE_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    batch = std::min(batch, n);
    const int32_t steps = (n + batch - 1) / batch;
    try {
        mlp->reserve(batch);
        if (mlp->perm_cap < n) {
            if (mlp->perm) cudaFree(mlp->perm);
            mlp->perm = nullptr;
            MC(cudaMalloc(&mlp->perm, sizeof(int32_t) * n));
            mlp->perm_cap = n;
        }
        if (mlp->loss_cap < steps) {
            if (mlp->loss) cudaFree(mlp->loss);
            mlp->loss = nullptr;
            MC(cudaMalloc(&mlp->loss, sizeof(float) * std::max(steps, 1024)));
            mlp->loss_cap = std::max(steps, 1024);
        }
        std::vector<int32_t> perm(n);
        std::vector<float> losses(steps, 0.f);
        uint64_t s = seed;
        for (int32_t e = 0; e < epochs; ++e) {
            for (int32_t i = 0; i < n; ++i) perm[i] = i;
            for (int32_t i = n - 1; i > 0; --i) {          // Fisher-Yates
                const int32_t j = (int32_t)(splitmix64(s) % (uint64_t)(i + 1));
                std::swap(perm[i], perm[j]);
            }
            MC(cudaMemcpyAsync(mlp->perm, perm.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, st));
            for (int32_t k = 0; k < steps; ++k) {
                const int32_t r0 = k * batch, rows = std::min(batch, n - r0);
                ++g_launches;
                k_gather<<<grid1((int64_t)rows * NIN, 256), 256, 0, st>>>(d_x, d_t, mlp->perm + r0, rows, mlp->xb,
                                                                          mlp->tb);
                mlp->standardize(mlp->xb, rows, mlp->x, st);
                mlp->backward(rows, mlp->tb, mlp->loss + k, st);
                mlp->adam_step(lr, weight_decay, st);
            }
            // the host permutation buffer is rewritten next epoch: wait for the upload
            MC(cudaStreamSynchronize(st));
        }
        MC(cudaGetLastError());
        if (loss && epochs > 0) {
            MC(cudaMemcpyAsync(losses.data(), mlp->loss, sizeof(float) * steps, cudaMemcpyDeviceToHost, st));
            MC(cudaStreamSynchronize(st));
            double acc = 0;
            for (float v : losses) acc += v;
            *loss = (float)(acc / steps);
        }
    } catch (const mlp_error &e) {
        cudaGetLastError();
        return e.st;
    }
    return AE_OK;
}

}  // extern "C"
