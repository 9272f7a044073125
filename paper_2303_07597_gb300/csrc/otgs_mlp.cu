// otgs_mlp.cu -- the learned warm start (no counterpart in the paper): the
// per-sample input features of a problem and a 3-layer perceptron that maps
// them to initial duals, trained with Adam on solutions the solver produced.
//
// Features of a problem (one row of in_dim floats per sample, source rows
// first, then target columns; entries past 9 + 2d are zero):
//   source i of class l: [0, min_j c_ij, mean_j c_ij, softmin_0.02, softmin_0.1,
//                         g_l / m, wl_0.5, wl_1, wl_2, x_i (d), mu_l (d)]
//   target j:            [1, min_i c_ij, mean_i c_ij, softmin_0.02, softmin_0.1,
//                         g_k / m, wl_0.5, wl_1, wl_2, y_j (d), mu_k (d)]
// mu_l = mean source feature of class l, g_l its size, k = the non-empty
// class whose mean is nearest to y_j, softmin_tau(v) = -tau log mean exp(-v/tau),
// wl_s = the level L with sum [L - v]_+ = s gamma / m (rows; / n for columns):
// the sample's dual when the other side's duals are constant and only the
// squared-L2 part of the regulariser acts.
//
// Network (width H, in_dim K, both multiples of 16): Z1 = q(X) q(W1)^T + b1,
// A1 = relu(Z1), Z2 = q(A1) q(W2)^T + b2, A2 = relu(Z2), y = q(A2) q(w3) + b3,
// q = rounding to bfloat16 (the tensor-core operands); loss mean (y - t)^2.
// The GEMMs run on the tensor cores (mma.sync m16n8k16, bf16 operands, FP32
// accumulators); the backward pass feeds bf16 copies of dZ2 and dZ1 to the
// weight-gradient GEMMs and keeps the bias gradients in FP32.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "otgs.h"

namespace otgs {

#define FULLMASK 0xffffffffu

typedef __nv_bfloat16 bf16;

namespace {

thread_local std::string g_mlp_err;

constexpr int NSTAT = 9;
// Water levels by Newton's method from the right: f(L) = sum_k [L - v_k]_+ - w
// is convex, increasing and piecewise linear in L, and f(min + w) >= 0, so
// from there each step L <- L - f(L) / #{v_k < L} stays at or right of the
// root and lands on it once it reaches the linear piece that holds it (a few
// passes over the values instead of a bisection's thirty).
constexpr int NREF = 4;  // second-pass inputs: three water levels and the own prediction
constexpr int WL_NEWTON_MAX = 32;

// ================================================================ GEMM
// C[M x N] = A[M x K] . B[N x K]^T, A and B bf16 row-major with K
// contiguous (row strides lda, ldb: multiples of 8 elements, 16-byte aligned
// rows), K a multiple of 16.  A CTA computes a 64 x 64 tile with 4 warps
// (32 x 32 each: 2 x 4 tiles of m16n8), K in steps of 32 through shared
// memory.  Epilogue, in this order: + bias[n], * [Zmask[m, n] > 0], relu;
// stores: FP32 (ldc), bf16 (ld16) and bf16 transposed (out16t[n * ld16t + m]).
constexpr int GM = 64, GN = 64, GK = 32, GPAD = 8;

struct GemmArgs {
    const bf16* A;
    int64_t lda;
    const bf16* B;
    int64_t ldb;
    int M, N, K;
    const float* bias;   // [N] or NULL
    const float* zmask;  // [M x N] FP32 (row stride ldz) or NULL
    int64_t ldz;
    int relu;
    float* out32;        // or NULL
    int64_t ldc;
    bf16* out16;         // or NULL
    int64_t ld16;
    bf16* out16t;        // or NULL
    int64_t ld16t;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__global__ void __launch_bounds__(128) k_gemm_nt(const GemmArgs g)
{
    __shared__ __align__(16) bf16 As[GM][GK + GPAD];
    __shared__ __align__(16) bf16 Bs[GN][GK + GPAD];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp >> 1, wn = warp & 1;
    const int m0 = blockIdx.y * GM, n0 = blockIdx.x * GN;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 4; j++)
#pragma unroll
            for (int c = 0; c < 4; c++) acc[i][j][c] = 0.f;
    // each thread moves one row's 16 consecutive k of A and of B per step
    const int lr = tid >> 1, lk = (tid & 1) * 16;
    for (int k0 = 0; k0 < g.K; k0 += GK) {
        uint4 va[2], vb[2];
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int k = k0 + lk + 8 * h;
            va[h] = make_uint4(0u, 0u, 0u, 0u);
            vb[h] = make_uint4(0u, 0u, 0u, 0u);
            if (m0 + lr < g.M && k < g.K) va[h] = *reinterpret_cast<const uint4*>(g.A + (int64_t)(m0 + lr) * g.lda + k);
            if (n0 + lr < g.N && k < g.K) vb[h] = *reinterpret_cast<const uint4*>(g.B + (int64_t)(n0 + lr) * g.ldb + k);
        }
        __syncthreads();  // the previous step's fragments are read
#pragma unroll
        for (int h = 0; h < 2; h++) {
            *reinterpret_cast<uint4*>(&As[lr][lk + 8 * h]) = va[h];
            *reinterpret_cast<uint4*>(&Bs[lr][lk + 8 * h]) = vb[h];
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < GK; ks += 16) {
            uint32_t a[2][4], b[4][2];
#pragma unroll
            for (int mt = 0; mt < 2; mt++) {
                const bf16* p = &As[wm * 32 + mt * 16 + (lane & 15)][ks + (lane >> 4) * 8];
                asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                             : "=r"(a[mt][0]), "=r"(a[mt][1]), "=r"(a[mt][2]), "=r"(a[mt][3])
                             : "r"(smem_u32(p)));
            }
#pragma unroll
            for (int nt = 0; nt < 4; nt++) {
                const bf16* p = &Bs[wn * 32 + nt * 8 + (lane & 7)][ks + ((lane >> 3) & 1) * 8];
                asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0, %1}, [%2];"
                             : "=r"(b[nt][0]), "=r"(b[nt][1])
                             : "r"(smem_u32(p)));
            }
#pragma unroll
            for (int mt = 0; mt < 2; mt++)
#pragma unroll
                for (int nt = 0; nt < 4; nt++)
                    asm volatile(
                        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
                        "{%8, %9}, {%0, %1, %2, %3};"
                        : "+f"(acc[mt][nt][0]), "+f"(acc[mt][nt][1]), "+f"(acc[mt][nt][2]), "+f"(acc[mt][nt][3])
                        : "r"(a[mt][0]), "r"(a[mt][1]), "r"(a[mt][2]), "r"(a[mt][3]), "r"(b[nt][0]),
                          "r"(b[nt][1]));
        }
    }
    // epilogue: accumulator c (of 4) sits at row lane/4 (+8 for c >= 2), column 2 (lane % 4) + (c & 1)
#pragma unroll
    for (int mt = 0; mt < 2; mt++)
#pragma unroll
        for (int nt = 0; nt < 4; nt++)
#pragma unroll
            for (int c = 0; c < 4; c++) {
                const int r = m0 + wm * 32 + mt * 16 + (lane >> 2) + (c >= 2 ? 8 : 0);
                const int col = n0 + wn * 32 + nt * 8 + (lane & 3) * 2 + (c & 1);
                if (r >= g.M || col >= g.N) continue;
                float v = acc[mt][nt][c];
                if (g.bias) v += g.bias[col];
                if (g.zmask && !(g.zmask[(int64_t)r * g.ldz + col] > 0.f)) v = 0.f;
                if (g.relu) v = fmaxf(v, 0.f);
                if (g.out32) g.out32[(int64_t)r * g.ldc + col] = v;
                if (g.out16) g.out16[(int64_t)r * g.ld16 + col] = __float2bfloat16_rn(v);
                if (g.out16t) g.out16t[(int64_t)col * g.ld16t + r] = __float2bfloat16_rn(v);
            }
}

void gemm(const GemmArgs& a, cudaStream_t st)
{
    dim3 grid((a.N + GN - 1) / GN, (a.M + GM - 1) / GM);
    k_gemm_nt<<<grid, 128, 0, st>>>(a);
}

// =========================================================== elementwise
// bf16 copy of an FP32 matrix [rows x cols] (ld_in), and optionally its
// transpose (outT[c * ldT + r]).
__global__ void k_to_bf16(const float* __restrict__ in, int64_t ld_in, int rows, int cols, bf16* out, int64_t ld_out,
                          bf16* outT, int64_t ldT)
{
    const int64_t n = (int64_t)rows * cols;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(q / cols), c = (int)(q % cols);
        const bf16 v = __float2bfloat16_rn(in[(int64_t)r * ld_in + c]);
        if (out) out[(int64_t)r * ld_out + c] = v;
        if (outT) outT[(int64_t)c * ldT + r] = v;
    }
}

void to_bf16(const float* in, int64_t ld_in, int rows, int cols, bf16* out, int64_t ld_out, bf16* outT, int64_t ldT,
             cudaStream_t st)
{
    const int64_t n = (int64_t)rows * cols;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
    k_to_bf16<<<blocks > 0 ? blocks : 1, 256, 0, st>>>(in, ld_in, rows, cols, out, ld_out, outT, ldT);
}

// Head of the network, one warp per sample: y = A2 . w3 + b3 (lanes take
// columns lane, lane + 32, ...; a fixed shuffle tree adds them).  With
// targets: dy = 2 (y - t) / B, r2 = (y - t)^2 and dZ2 = dy w3 * [Z2 > 0] as
// FP32, bf16 and transposed bf16.
__global__ void k_head(const bf16* __restrict__ A2, const float* __restrict__ Z2, int H, int Bn,
                       const bf16* __restrict__ w3, const float* b3, const float* __restrict__ t, float* y, float* dy,
                       float* r2, float* dZ2, bf16* dZ2b, bf16* dZ2t, int64_t ldt)
{
    const int lane = threadIdx.x & 31;
    const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (b >= Bn) return;
    float s = 0.f;
    for (int h = lane; h < H; h += 32)
        s = fmaf(__bfloat162float(A2[(int64_t)b * H + h]), __bfloat162float(w3[h]), s);
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) s += __shfl_xor_sync(FULLMASK, s, off);
    const float yb = s + b3[0];
    if (lane == 0) y[b] = yb;
    if (!t) return;
    const float r = yb - t[b];
    const float d = 2.f * r / (float)Bn;
    if (lane == 0) {
        dy[b] = d;
        r2[b] = r * r;
    }
    for (int h = lane; h < H; h += 32) {
        const float v = Z2[(int64_t)b * H + h] > 0.f ? d * __bfloat162float(w3[h]) : 0.f;
        dZ2[(int64_t)b * H + h] = v;
        const bf16 vb = __float2bfloat16_rn(v);
        dZ2b[(int64_t)b * H + h] = vb;
        dZ2t[(int64_t)h * ldt + b] = vb;
    }
}

// out[c] = sum_r w[r] M[r, c] (w = 1 when NULL), rows added in order per
// thread group and the 8 groups in order: deterministic.  M is FP32 or bf16.
template <class T>
__global__ void __launch_bounds__(256) k_colsum(const T* __restrict__ M, int64_t ld, int rows, int cols,
                                                const float* __restrict__ w, float* out)
{
    __shared__ float part[8][32];
    const int c = blockIdx.x * 32 + (threadIdx.x & 31), grp = threadIdx.x >> 5;
    float s = 0.f;
    if (c < cols)
        for (int r = grp; r < rows; r += 8) {
            const float v = (float)M[(int64_t)r * ld + c];
            s = w ? fmaf(w[r], v, s) : s + v;
        }
    part[grp][threadIdx.x & 31] = s;
    __syncthreads();
    if (grp == 0 && c < cols) {
        float t = 0.f;
        for (int q = 0; q < 8; q++) t += part[q][threadIdx.x & 31];
        out[c] = t;
    }
}

template <class T>
void colsum(const T* M, int64_t ld, int rows, int cols, const float* w, float* out, cudaStream_t st)
{
    k_colsum<T><<<(cols + 31) / 32, 256, 0, st>>>(M, ld, rows, cols, w, out);
}

__global__ void k_scale(float* v, float s) { v[0] *= s; }

// Adam on the FP32 parameters (bias-corrected moments).
__global__ void k_adam(float* p, const float* __restrict__ g, float* m1, float* m2, int64_t n, float lr, float b1,
                       float b2, float eps, float c1, float c2)
{
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const float gv = g[q];
        const float m = b1 * m1[q] + (1.f - b1) * gv;
        const float v = b2 * m2[q] + (1.f - b2) * gv * gv;
        m1[q] = m;
        m2[q] = v;
        p[q] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
    }
}

// Initial weights: uniform in [-a, a] (a = sqrt(6 / fan_in), He et al. 2015)
// from SplitMix64 (Steele, Lea and Flood, 2014) of (seed, index); biases 0.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x)
{
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

__global__ void k_init(float* p, int64_t n, int64_t w1, int64_t b1e, int64_t w2e, int64_t b2e, int64_t w3e, int K, int H,
                       uint64_t seed)
{
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const double u = (double)(splitmix64(seed * 0x100000001B3ull + (uint64_t)q) >> 11) * 0x1p-53;  // [0, 1)
        float a = 0.f;
        if (q < w1) a = sqrtf(6.f / (float)K);
        else if (q >= b1e && q < w2e) a = sqrtf(6.f / (float)H);
        else if (q >= b2e && q < w3e) a = sqrtf(3.f / (float)H);
        p[q] = (float)((2.0 * u - 1.0) * a);
    }
}

// ============================================================= features
// Statistics of a cost row or column: min, mean, softmin for the two
// temperatures and the water levels of masses w * {0.5, 1, 2}, over `cnt`
// values at stride `stride` (FP32, in order).
__device__ __forceinline__ void cost_stats(const float* v, int64_t stride, int cnt, float w, float* out)
{
    float mn = INFINITY;
    double sum = 0.0;
    for (int k = 0; k < cnt; k++) {
        const float c = v[(int64_t)k * stride];
        mn = fminf(mn, c);
        sum += (double)c;
    }
    float e1 = 0.f, e2 = 0.f;
    for (int k = 0; k < cnt; k++) {
        const float c = v[(int64_t)k * stride] - mn;
        e1 += expf(-c / 0.02f);
        e2 += expf(-c / 0.1f);
    }
    out[0] = mn;
    out[1] = (float)(sum / (double)cnt);
    out[2] = mn - 0.02f * logf(e1 / (float)cnt);
    out[3] = mn - 0.1f * logf(e2 / (float)cnt);
    const float mass[3] = {0.5f * w, w, 2.f * w};
#pragma unroll
    for (int q = 0; q < 3; q++) {
        float L = mn + mass[q];
        for (int it = 0; it < WL_NEWTON_MAX; it++) {
            float sum = 0.f, below = 0.f;
            for (int k = 0; k < cnt; k++) {
                const float dl = L - v[(int64_t)k * stride];
                if (dl > 0.f) {
                    sum += dl;
                    below += 1.f;
                }
            }
            const float f = sum - mass[q];
            if (!(f > 0.f)) break;  // at the root (or just left of it, by rounding)
            const float Ln = L - f / below;
            if (!(Ln < L)) break;
            L = Ln;
        }
        out[4 + q] = L;
    }
}

// Batched features: problem table entries.
struct FeatProb {
    const float* C;
    const float* XS;
    const float* XT;
    const int32_t* lab;
    int64_t ldc;
    int32_t m, n, L;
    int32_t roff, coff;  // first source row / target column in the concatenation
    int32_t moff;        // first class of the problem in the class-mean table
};

// Class means of every problem: one CTA per problem, a thread per (class,
// feature) pair walking the problem's rows in order (FP64 sums).
__global__ void __launch_bounds__(256) k_class_means_b(const FeatProb* __restrict__ P, int d, float* mu, int* gsz)
{
    const FeatProb p = P[blockIdx.x];
    for (int q = threadIdx.x; q < p.L * d; q += blockDim.x) {
        const int l = q / d, c = q % d;
        double s = 0.0;
        int cnt = 0;
        // rows in order, eight labels (and their rows' values) loaded ahead
        for (int i0 = 0; i0 < p.m; i0 += 8) {
            int lb[8];
#pragma unroll
            for (int u = 0; u < 8; u++) lb[u] = i0 + u < p.m ? __ldg(p.lab + i0 + u) : -1;
            float xv[8];
#pragma unroll
            for (int u = 0; u < 8; u++) xv[u] = lb[u] == l ? __ldg(p.XS + (int64_t)(i0 + u) * d + c) : 0.f;
#pragma unroll
            for (int u = 0; u < 8; u++)
                if (lb[u] == l) {
                    s += (double)xv[u];
                    cnt++;
                }
        }
        mu[(int64_t)(p.moff + l) * d + c] = cnt ? (float)(s / cnt) : 0.f;
        if (c == 0) gsz[p.moff + l] = cnt;
    }
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(FULLMASK, v, off);
    return v;
}

// The statistics of cost_stats for one contiguous row, a warp at a time
// (lanes take every 32nd value; the same in every lane on return).
__device__ __forceinline__ void row_stats_warp(const float* v, int cnt, float w, float* out)
{
    const int lane = threadIdx.x & 31;
    float mn = INFINITY;
    double sum = 0.0;
    for (int k = lane; k < cnt; k += 32) {
        const float c = v[k];
        mn = fminf(mn, c);
        sum += (double)c;
    }
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        mn = fminf(mn, __shfl_xor_sync(FULLMASK, mn, off));
        sum += __shfl_xor_sync(FULLMASK, sum, off);
    }
    float e1 = 0.f, e2 = 0.f;
    for (int k = lane; k < cnt; k += 32) {
        const float c = v[k] - mn;
        e1 += expf(-c / 0.02f);
        e2 += expf(-c / 0.1f);
    }
    e1 = warp_sum(e1);
    e2 = warp_sum(e2);
    out[0] = mn;
    out[1] = (float)(sum / (double)cnt);
    out[2] = mn - 0.02f * logf(e1 / (float)cnt);
    out[3] = mn - 0.1f * logf(e2 / (float)cnt);
    const float mass[3] = {0.5f * w, w, 2.f * w};
#pragma unroll
    for (int q = 0; q < 3; q++) {
        float L = mn + mass[q];  // Newton from the right, as in cost_stats (the same in every lane)
        for (int it = 0; it < WL_NEWTON_MAX; it++) {
            float part = 0.f, below = 0.f;
            for (int k = lane; k < cnt; k += 32) {
                const float dl = L - v[k];
                if (dl > 0.f) {
                    part += dl;
                    below += 1.f;
                }
            }
            const float f = warp_sum(part) - mass[q];
            below = warp_sum(below);
            if (!(f > 0.f)) break;
            const float Ln = L - f / below;
            if (!(Ln < L)) break;
            L = Ln;
        }
        out[4 + q] = L;
    }
}

// The problem holding global row (src) or column index g (offsets increase).
__device__ __forceinline__ int find_prob(const FeatProb* __restrict__ P, int nprob, bool src, int64_t g)
{
    int lo = 0, hi = nprob - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((src ? P[mid].roff : P[mid].coff) <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Source samples, one warp each: rows [0, M) of the output.
__global__ void k_features_src(const FeatProb* __restrict__ P, int nprob, int64_t Mtot, int d,
                               const float* __restrict__ mu, const int* __restrict__ gsz, float gamma, int in_dim,
                               float* out)
{
    const int lane = threadIdx.x & 31;
    const int64_t g = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (g >= Mtot) return;
    const FeatProb p = P[find_prob(P, nprob, true, g)];
    const int i = (int)(g - p.roff);
    float st[7];
    row_stats_warp(p.C + (int64_t)i * p.ldc, p.n, gamma / (float)p.m, st);
    int cls = p.lab[i];
    if (cls < 0 || cls >= p.L) cls = -1;  // an invalid label: no class entries
    float* o = out + g * in_dim;
    const float* x = p.XS + (int64_t)i * d;
    const float* mup = mu + (int64_t)(p.moff + (cls >= 0 ? cls : 0)) * d;
    if (lane == 0) {
        o[0] = 0.f;
        for (int q = 0; q < 4; q++) o[1 + q] = st[q];
        o[5] = cls >= 0 ? (float)gsz[p.moff + cls] / (float)p.m : 0.f;
        for (int q = 0; q < 3; q++) o[6 + q] = st[4 + q];
    }
    for (int c = lane; c < d; c += 32) {
        o[NSTAT + c] = x[c];
        o[NSTAT + d + c] = cls >= 0 ? mup[c] : 0.f;
    }
    for (int c = NSTAT + 2 * d + lane; c < in_dim; c += 32) o[c] = 0.f;
}

// Target samples, one thread each (a column's values are read coalesced
// across the threads): rows [M, M + N) of the output.
__global__ void k_features_tgt(const FeatProb* __restrict__ P, int nprob, int64_t Mtot, int64_t Ntot, int d,
                               const float* __restrict__ mu, const int* __restrict__ gsz, float gamma, int in_dim,
                               float* out)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= Ntot) return;
    const int64_t q = Mtot + g;
    const FeatProb p = P[find_prob(P, nprob, false, g)];
    float* o = out + q * in_dim;
    float st[7];
    int cls;
    const float* x;
    const float* mup = mu + (int64_t)p.moff * d;
    const int* gz = gsz + p.moff;
    {
        const int j = (int)(g - p.coff);
        cost_stats(p.C + j, p.ldc, p.m, gamma / (float)p.n, st);
        x = p.XT + (int64_t)j * d;
        float best = INFINITY;
        cls = -1;
        for (int l = 0; l < p.L; l++) {
            if (gz[l] == 0) continue;
            float dist = 0.f;
            for (int c = 0; c < d; c++) {
                const float df = __fsub_rn(x[c], mup[(int64_t)l * d + c]);
                dist = __fadd_rn(dist, __fmul_rn(df, df));
            }
            if (dist < best) {
                best = dist;
                cls = l;
            }
        }
        o[0] = 1.f;
    }
    o[1] = st[0];
    o[2] = st[1];
    o[3] = st[2];
    o[4] = st[3];
    o[5] = cls >= 0 ? (float)gz[cls] / (float)p.m : 0.f;
    o[6] = st[4];
    o[7] = st[5];
    o[8] = st[6];
    for (int c = 0; c < d; c++) {
        o[NSTAT + c] = x[c];
        o[NSTAT + d + c] = cls >= 0 ? mup[(int64_t)cls * d + c] : 0.f;
    }
    for (int c = NSTAT + 2 * d; c < in_dim; c++) o[c] = 0.f;
}

// ------------------------------------------------------- second pass
// Water level of the values v_k - o_k (k < cnt; v at stride `stride`), by
// the Newton steps of cost_stats, one thread.
__device__ __forceinline__ float wl_shifted_thread(const float* v, int64_t stride, const float* o, int cnt, float mn,
                                                   float mass)
{
    float L = mn + mass;
    for (int it = 0; it < WL_NEWTON_MAX; it++) {
        float sum = 0.f, below = 0.f;
        for (int k = 0; k < cnt; k++) {
            const float dl = L - __fsub_rn(v[(int64_t)k * stride], o[k]);
            if (dl > 0.f) {
                sum += dl;
                below += 1.f;
            }
        }
        const float f = sum - mass;
        if (!(f > 0.f)) break;
        const float Ln = L - f / below;
        if (!(Ln < L)) break;
        L = Ln;
    }
    return L;
}

// The same for one contiguous row, a warp at a time (the same in every lane).
__device__ __forceinline__ float wl_shifted_warp(const float* v, const float* o, int cnt, float mn, float mass)
{
    const int lane = threadIdx.x & 31;
    float L = mn + mass;
    for (int it = 0; it < WL_NEWTON_MAX; it++) {
        float part = 0.f, below = 0.f;
        for (int k = lane; k < cnt; k += 32) {
            const float dl = L - __fsub_rn(v[k], o[k]);
            if (dl > 0.f) {
                part += dl;
                below += 1.f;
            }
        }
        const float f = warp_sum(part) - mass;
        below = warp_sum(below);
        if (!(f > 0.f)) break;
        const float Ln = L - f / below;
        if (!(Ln < L)) break;
        L = Ln;
    }
    return L;
}

// Second-pass inputs of source rows, one warp each: the water levels of
// c_ij - beta_hat_j over the problem's columns, and alpha_hat_i, into
// columns [col0, col0 + 4) of the row's features.
__global__ void k_refine_src(const FeatProb* __restrict__ P, int nprob, int64_t Mtot, const float* __restrict__ ahat,
                             const float* __restrict__ bhat, float gamma, int col0, int in_dim, float* out)
{
    const int lane = threadIdx.x & 31;
    const int64_t g = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (g >= Mtot) return;
    const FeatProb p = P[find_prob(P, nprob, true, g)];
    const int i = (int)(g - p.roff);
    const float* v = p.C + (int64_t)i * p.ldc;
    const float* o = bhat + p.coff;
    float mn = INFINITY;
    for (int k = lane; k < p.n; k += 32) mn = fminf(mn, __fsub_rn(v[k], o[k]));
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) mn = fminf(mn, __shfl_xor_sync(FULLMASK, mn, off));
    const float w = gamma / (float)p.m;
    const float l0 = wl_shifted_warp(v, o, p.n, mn, 0.5f * w);
    const float l1 = wl_shifted_warp(v, o, p.n, mn, w);
    const float l2 = wl_shifted_warp(v, o, p.n, mn, 2.f * w);
    if (lane == 0) {
        float* q = out + g * in_dim + col0;
        q[0] = l0;
        q[1] = l1;
        q[2] = l2;
        q[3] = ahat[g];
    }
}

// Second-pass inputs of target columns, one thread each: the water levels
// of c_ij - alpha_hat_i over the problem's rows, and beta_hat_j.
__global__ void k_refine_tgt(const FeatProb* __restrict__ P, int nprob, int64_t Mtot, int64_t Ntot,
                             const float* __restrict__ ahat, const float* __restrict__ bhat, float gamma, int col0,
                             int in_dim, float* out)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= Ntot) return;
    const FeatProb p = P[find_prob(P, nprob, false, g)];
    const int j = (int)(g - p.coff);
    const float* v = p.C + j;
    const float* o = ahat + p.roff;
    float mn = INFINITY;
    for (int k = 0; k < p.m; k++) mn = fminf(mn, __fsub_rn(v[(int64_t)k * p.ldc], o[k]));
    const float w = gamma / (float)p.n;
    float* q = out + (Mtot + g) * in_dim + col0;
    q[0] = wl_shifted_thread(v, p.ldc, o, p.m, mn, 0.5f * w);
    q[1] = wl_shifted_thread(v, p.ldc, o, p.m, mn, w);
    q[2] = wl_shifted_thread(v, p.ldc, o, p.m, mn, 2.f * w);
    q[3] = bhat[g];
}

}  // namespace

// ================================================================ handle
struct Mlp {
    int K = 0, H = 0;
    int64_t cap = 0, capp = 0;  // batch capacity; rounded up to 16 (transposed operands' row stride)
    cudaStream_t st = nullptr;
    std::vector<void*> allocs;
    std::string err;
    int64_t np = 0;                 // parameters
    int64_t o_b1, o_W2, o_b2, o_w3, o_b3;
    float *P = nullptr, *G = nullptr, *M1 = nullptr, *M2 = nullptr;
    bf16 *W1b = nullptr, *W2b = nullptr, *W2t = nullptr, *w3b = nullptr;
    bf16 *Xb = nullptr, *Xt = nullptr, *A1b = nullptr, *A1t = nullptr, *A2b = nullptr;
    bf16 *dZ2b = nullptr, *dZ2t = nullptr, *dZ1t = nullptr;
    float *Z1 = nullptr, *Z2 = nullptr;  // A1, A2 in FP32 ([A > 0] = [Z > 0]: the backward masks)
    float *y = nullptr, *dy = nullptr, *r2 = nullptr, *dZ2 = nullptr, *dZ1 = nullptr;
    bool failed = false;                  // an allocation failed
    long long step = 0;
    bool have_grad = false;
    ~Mlp()
    {
        for (void* p : allocs) cudaFree(p);
    }
    void* al(size_t bytes)
    {
        void* p = nullptr;
        if (cudaMalloc(&p, bytes ? bytes : 16) != cudaSuccess) {
            cudaGetLastError();
            failed = true;
            return nullptr;
        }
        allocs.push_back(p);
        return p;
    }
    bool ck(cudaError_t e, const char* what)
    {
        if (e == cudaSuccess) return true;
        err = std::string(what) + ": " + cudaGetErrorString(e);
        return false;
    }
    // bf16 copies of the weights (and W2 transposed)
    void weights_bf16()
    {
        to_bf16(P, K, H, K, W1b, K, nullptr, 0, st);
        to_bf16(P + o_W2, H, H, H, W2b, H, W2t, H, st);
        to_bf16(P + o_w3, H, 1, H, w3b, H, nullptr, 0, st);
    }
    void forward(const float* X, int Bn, bool train);
};

void Mlp::forward(const float* X, int Bn, bool train)
{
    to_bf16(X, K, Bn, K, Xb, K, train ? Xt : nullptr, capp, st);
    // A1 = relu(X W1^T + b1): FP32 (the backward pass's mask), bf16 (and transposed)
    GemmArgs g;
    memset(&g, 0, sizeof(g));
    g.A = Xb; g.lda = K; g.B = W1b; g.ldb = K; g.M = Bn; g.N = H; g.K = K;
    g.bias = P + o_b1; g.relu = 1; g.out32 = Z1; g.ldc = H; g.out16 = A1b; g.ld16 = H;
    if (train) { g.out16t = A1t; g.ld16t = capp; }
    gemm(g, st);
    // A2 = relu(A1 W2^T + b2)
    memset(&g, 0, sizeof(g));
    g.A = A1b; g.lda = H; g.B = W2b; g.ldb = H; g.M = Bn; g.N = H; g.K = H;
    g.bias = P + o_b2; g.relu = 1; g.out32 = Z2; g.ldc = H; g.out16 = A2b; g.ld16 = H;
    gemm(g, st);
}

}  // namespace otgs

using namespace otgs;

struct ot_gs_mlp {
    Mlp m;
};

extern "C" {

const char* ot_gs_mlp_last_error(const ot_gs_mlp* h) { return h ? h->m.err.c_str() : g_mlp_err.c_str(); }

int ot_gs_mlp_create(ot_gs_mlp** out, int32_t in_dim, int32_t width, int64_t max_batch, uint64_t seed, void* stream)
{
    g_mlp_err.clear();
    if (!out) { g_mlp_err = "h is NULL"; return OTGS_EINVAL; }
    *out = nullptr;
    if (in_dim <= 0 || in_dim % 16 || width <= 0 || width % 16 || max_batch <= 0 || max_batch > (1 << 24)) {
        g_mlp_err = "need in_dim, width > 0 multiples of 16 and 0 < max_batch <= 2^24";
        return OTGS_EINVAL;
    }
    ot_gs_mlp* h = new (std::nothrow) ot_gs_mlp();
    if (!h) { g_mlp_err = "out of host memory"; return OTGS_ENOMEM; }
    Mlp& M = h->m;
    M.K = in_dim;
    M.H = width;
    M.cap = max_batch;
    M.capp = (max_batch + 15) / 16 * 16;
    M.st = (cudaStream_t)stream;
    const int64_t K = in_dim, H = width;
    M.o_b1 = H * K;
    M.o_W2 = M.o_b1 + H;
    M.o_b2 = M.o_W2 + H * H;
    M.o_w3 = M.o_b2 + H;
    M.o_b3 = M.o_w3 + H;
    M.np = M.o_b3 + 1;
    const size_t fb = sizeof(float) * (size_t)M.np;
    M.P = (float*)M.al(fb);
    M.G = (float*)M.al(fb);
    M.M1 = (float*)M.al(fb);
    M.M2 = (float*)M.al(fb);
    M.W1b = (bf16*)M.al(2 * (size_t)(H * K));
    M.W2b = (bf16*)M.al(2 * (size_t)(H * H));
    M.W2t = (bf16*)M.al(2 * (size_t)(H * H));
    M.w3b = (bf16*)M.al(2 * (size_t)H);
    const size_t cb = (size_t)M.cap, cp = (size_t)M.capp;
    M.Xb = (bf16*)M.al(2 * cb * K);
    M.Xt = (bf16*)M.al(2 * cp * K);
    M.A1b = (bf16*)M.al(2 * cb * H);
    M.A1t = (bf16*)M.al(2 * cp * H);
    M.A2b = (bf16*)M.al(2 * cb * H);
    M.dZ2b = (bf16*)M.al(2 * cb * H);
    M.dZ2t = (bf16*)M.al(2 * cp * H);
    M.dZ1t = (bf16*)M.al(2 * cp * H);
    M.Z1 = (float*)M.al(4 * cb * H);
    M.Z2 = (float*)M.al(4 * cb * H);
    M.dZ2 = (float*)M.al(4 * cb * H);
    M.dZ1 = (float*)M.al(4 * cb * H);
    M.y = (float*)M.al(4 * cb);
    M.dy = (float*)M.al(4 * cb);
    M.r2 = (float*)M.al(4 * cb);
    if (M.failed) {
        g_mlp_err = "cudaMalloc failed";
        delete h;
        return OTGS_ENOMEM;
    }
    k_init<<<256, 256, 0, M.st>>>(M.P, M.np, M.o_b1, M.o_b1, M.o_W2, M.o_b2, M.o_w3, (int)K, (int)H, seed);
    // the biases and b3 are zero: k_init gives 0 outside the weight ranges
    cudaMemsetAsync(M.M1, 0, fb, M.st);
    cudaMemsetAsync(M.M2, 0, fb, M.st);
    M.weights_bf16();
    if (!M.ck(cudaGetLastError(), "mlp init") || !M.ck(cudaStreamSynchronize(M.st), "mlp init")) {
        g_mlp_err = M.err;
        delete h;
        return OTGS_ECUDA;
    }
    *out = h;
    return OTGS_OK;
}

int ot_gs_mlp_destroy(ot_gs_mlp* h)
{
    if (!h) return OTGS_OK;
    cudaStreamSynchronize(h->m.st);
    delete h;
    return OTGS_OK;
}

int ot_gs_mlp_num_params(const ot_gs_mlp* h, int64_t* n)
{
    if (!h || !n) return OTGS_EINVAL;
    *n = h->m.np;
    return OTGS_OK;
}

int ot_gs_mlp_set_params(ot_gs_mlp* h, const float* p)
{
    if (!h || !p) return OTGS_EINVAL;
    Mlp& M = h->m;
    if (!M.ck(cudaMemcpyAsync(M.P, p, sizeof(float) * M.np, cudaMemcpyDeviceToDevice, M.st), "set_params"))
        return OTGS_ECUDA;
    cudaMemsetAsync(M.M1, 0, sizeof(float) * M.np, M.st);
    cudaMemsetAsync(M.M2, 0, sizeof(float) * M.np, M.st);
    M.step = 0;
    M.have_grad = false;
    M.weights_bf16();
    return M.ck(cudaGetLastError(), "set_params") ? OTGS_OK : OTGS_ECUDA;
}

int ot_gs_mlp_get_params(ot_gs_mlp* h, float* p)
{
    if (!h || !p) return OTGS_EINVAL;
    Mlp& M = h->m;
    return M.ck(cudaMemcpyAsync(p, M.P, sizeof(float) * M.np, cudaMemcpyDeviceToDevice, M.st), "get_params")
               ? OTGS_OK
               : OTGS_ECUDA;
}

int ot_gs_mlp_forward(ot_gs_mlp* h, const float* X, int64_t B, float* y)
{
    if (!h) return OTGS_EINVAL;
    Mlp& M = h->m;
    if (!X || !y || B <= 0 || B > M.cap) {
        M.err = "need X, y and 0 < B <= max_batch";
        return OTGS_EINVAL;
    }
    M.forward(X, (int)B, false);
    const int wpb = 8;
    k_head<<<(int)((B + wpb - 1) / wpb), 32 * wpb, 0, M.st>>>(M.A2b, M.Z2, M.H, (int)B, M.w3b, M.P + M.o_b3, nullptr, y,
                                                              nullptr, nullptr, nullptr, nullptr, nullptr, 0);
    return M.ck(cudaGetLastError(), "mlp forward") ? OTGS_OK : OTGS_ECUDA;
}

int ot_gs_mlp_grad(ot_gs_mlp* h, const float* X, const float* t, int64_t B, float* loss, float* grad)
{
    if (!h) return OTGS_EINVAL;
    Mlp& M = h->m;
    if (!X || !t || B <= 0 || B > M.cap) {
        M.err = "need X, t and 0 < B <= max_batch";
        return OTGS_EINVAL;
    }
    const int Bn = (int)B, H = M.H, K = M.K;
    cudaStream_t st = M.st;
    // transposed operands: columns past B must be zero (they enter the weight-gradient sums)
    cudaMemsetAsync(M.Xt, 0, 2 * (size_t)M.capp * K, st);
    cudaMemsetAsync(M.A1t, 0, 2 * (size_t)M.capp * H, st);
    cudaMemsetAsync(M.dZ2t, 0, 2 * (size_t)M.capp * H, st);
    cudaMemsetAsync(M.dZ1t, 0, 2 * (size_t)M.capp * H, st);
    M.forward(X, Bn, true);
    const int wpb = 8;
    k_head<<<(Bn + wpb - 1) / wpb, 32 * wpb, 0, st>>>(M.A2b, M.Z2, H, Bn, M.w3b, M.P + M.o_b3, t, M.y, M.dy, M.r2,
                                                      M.dZ2, M.dZ2b, M.dZ2t, M.capp);
    float* G = M.G;
    // g_w3 = A2^T dy, g_b3 = sum dy, g_b2 = sum_b dZ2
    colsum<bf16>(M.A2b, H, Bn, H, M.dy, G + M.o_w3, st);
    colsum<float>(M.dy, 1, Bn, 1, nullptr, G + M.o_b3, st);
    colsum<float>(M.dZ2, H, Bn, H, nullptr, G + M.o_b2, st);
    // dZ1 = (dZ2 W2) * [Z1 > 0]
    GemmArgs g;
    memset(&g, 0, sizeof(g));
    g.A = M.dZ2b; g.lda = H; g.B = M.W2t; g.ldb = H; g.M = Bn; g.N = H; g.K = H;
    g.zmask = M.Z1; g.ldz = H; g.out32 = M.dZ1; g.ldc = H; g.out16t = M.dZ1t; g.ld16t = M.capp;
    gemm(g, st);
    colsum<float>(M.dZ1, H, Bn, H, nullptr, G + M.o_b1, st);
    // g_W2 = dZ2^T A1, g_W1 = dZ1^T X (sums over the batch)
    const int Kb = (int)((Bn + 15) / 16 * 16);
    memset(&g, 0, sizeof(g));
    g.A = M.dZ2t; g.lda = M.capp; g.B = M.A1t; g.ldb = M.capp; g.M = H; g.N = H; g.K = Kb;
    g.out32 = G + M.o_W2; g.ldc = H;
    gemm(g, st);
    memset(&g, 0, sizeof(g));
    g.A = M.dZ1t; g.lda = M.capp; g.B = M.Xt; g.ldb = M.capp; g.M = H; g.N = K; g.K = Kb;
    g.out32 = G; g.ldc = K;
    gemm(g, st);
    if (loss) {
        colsum<float>(M.r2, 1, Bn, 1, nullptr, loss, st);  // sum of squares
        k_scale<<<1, 1, 0, st>>>(loss, 1.f / (float)Bn);
    }
    if (grad && !M.ck(cudaMemcpyAsync(grad, G, sizeof(float) * M.np, cudaMemcpyDeviceToDevice, st), "grad copy"))
        return OTGS_ECUDA;
    M.have_grad = true;
    return M.ck(cudaGetLastError(), "mlp grad") ? OTGS_OK : OTGS_ECUDA;
}

int ot_gs_mlp_adam(ot_gs_mlp* h, float lr, float b1, float b2, float eps)
{
    if (!h) return OTGS_EINVAL;
    Mlp& M = h->m;
    if (!M.have_grad) {
        M.err = "no gradient: call ot_gs_mlp_grad first";
        return OTGS_EINVAL;
    }
    M.step++;
    const float c1 = 1.f - powf(b1, (float)M.step), c2 = 1.f - powf(b2, (float)M.step);
    k_adam<<<(int)std::min<int64_t>((M.np + 255) / 256, 2048), 256, 0, M.st>>>(M.P, M.G, M.M1, M.M2, M.np, lr, b1, b2,
                                                                              eps, c1, c2);
    M.weights_bf16();
    return M.ck(cudaGetLastError(), "mlp adam") ? OTGS_OK : OTGS_ECUDA;
}

int ot_gs_mlp_features(const float* C, int64_t ldc, int64_t m, int64_t n, const float* XS, const float* XT,
                       int32_t d, const int32_t* labels, int32_t L, float gamma, int32_t in_dim, float* out,
                       void* stream)
{
    return ot_gs_mlp_features_batch(1, &C, &ldc, &m, &n, &XS, &XT, d, &labels, &L, gamma, in_dim, out, stream);
}

int ot_gs_mlp_features_batch(int32_t nprob, const float* const* C, const int64_t* ldc, const int64_t* m,
                             const int64_t* n, const float* const* XS, const float* const* XT, int32_t d,
                             const int32_t* const* labels, const int32_t* L, float gamma, int32_t in_dim,
                             float* out, void* stream)
{
    g_mlp_err.clear();
    if (nprob <= 0 || !C || !ldc || !m || !n || !XS || !XT || !labels || !L || !out || d <= 0 ||
        in_dim < NSTAT + 2 * d || !(gamma > 0.f)) {
        g_mlp_err = "invalid batched features arguments (in_dim >= 9 + 2 d, gamma > 0)";
        return OTGS_EINVAL;
    }
    std::vector<FeatProb> tab(nprob);
    int64_t M = 0, N = 0, LL = 0;
    for (int32_t k = 0; k < nprob; k++) {
        if (!C[k] || !XS[k] || !XT[k] || !labels[k] || m[k] <= 0 || n[k] <= 0 || L[k] <= 0 || ldc[k] < n[k]) {
            g_mlp_err = "invalid problem " + std::to_string(k);
            return OTGS_EINVAL;
        }
        FeatProb& p = tab[k];
        p.C = C[k]; p.XS = XS[k]; p.XT = XT[k]; p.lab = labels[k]; p.ldc = ldc[k];
        p.m = (int32_t)m[k]; p.n = (int32_t)n[k]; p.L = L[k];
        p.roff = (int32_t)M; p.coff = (int32_t)N; p.moff = (int32_t)LL;
        M += m[k];
        N += n[k];
        LL += L[k];
        if (M > INT32_MAX / 2 || N > INT32_MAX / 2 || LL * d > INT32_MAX / 2) {
            g_mlp_err = "batch too large";
            return OTGS_EINVAL;
        }
    }
    cudaStream_t st = (cudaStream_t)stream;
    FeatProb* dtab = nullptr;
    float* mu = nullptr;
    int* gsz = nullptr;
    if (cudaMallocAsync(&dtab, sizeof(FeatProb) * (size_t)nprob, st) != cudaSuccess ||
        cudaMallocAsync(&mu, sizeof(float) * (size_t)(LL * d), st) != cudaSuccess ||
        cudaMallocAsync(&gsz, sizeof(int) * (size_t)LL, st) != cudaSuccess) {
        cudaGetLastError();
        if (dtab) cudaFreeAsync(dtab, st);
        if (mu) cudaFreeAsync(mu, st);
        g_mlp_err = "cudaMallocAsync failed";
        return OTGS_ENOMEM;
    }
    cudaMemcpyAsync(dtab, tab.data(), sizeof(FeatProb) * (size_t)nprob, cudaMemcpyHostToDevice, st);
    k_class_means_b<<<nprob, 256, 0, st>>>(dtab, d, mu, gsz);
    k_features_src<<<(int)((M + 7) / 8), 256, 0, st>>>(dtab, nprob, M, d, mu, gsz, gamma, in_dim, out);
    k_features_tgt<<<(int)((N + 127) / 128), 128, 0, st>>>(dtab, nprob, M, N, d, mu, gsz, gamma, in_dim, out);
    cudaFreeAsync(dtab, st);
    cudaFreeAsync(mu, st);
    cudaFreeAsync(gsz, st);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        g_mlp_err = std::string("batched features: ") + cudaGetErrorString(e);
        return OTGS_ECUDA;
    }
    return OTGS_OK;
}

int ot_gs_mlp_refine_features(int32_t nprob, const float* const* C, const int64_t* ldc, const int64_t* m,
                              const int64_t* n, const float* alpha_hat, const float* beta_hat, float gamma,
                              int32_t col0, int32_t in_dim, float* out, void* stream)
{
    g_mlp_err.clear();
    if (nprob <= 0 || !C || !ldc || !m || !n || !alpha_hat || !beta_hat || !out || !(gamma > 0.f) || col0 < 0 ||
        col0 > in_dim - NREF) {
        g_mlp_err = "invalid second-pass features arguments (0 <= col0 <= in_dim - 4, gamma > 0)";
        return OTGS_EINVAL;
    }
    std::vector<FeatProb> tab(nprob);
    int64_t M = 0, N = 0;
    for (int32_t k = 0; k < nprob; k++) {
        if (!C[k] || m[k] <= 0 || n[k] <= 0 || ldc[k] < n[k]) {
            g_mlp_err = "invalid problem " + std::to_string(k);
            return OTGS_EINVAL;
        }
        FeatProb& p = tab[k];
        p = FeatProb{};
        p.C = C[k]; p.ldc = ldc[k];
        p.m = (int32_t)m[k]; p.n = (int32_t)n[k];
        p.roff = (int32_t)M; p.coff = (int32_t)N;
        M += m[k];
        N += n[k];
        if (M > INT32_MAX / 2 || N > INT32_MAX / 2) {
            g_mlp_err = "batch too large";
            return OTGS_EINVAL;
        }
    }
    cudaStream_t st = (cudaStream_t)stream;
    FeatProb* dtab = nullptr;
    if (cudaMallocAsync(&dtab, sizeof(FeatProb) * (size_t)nprob, st) != cudaSuccess) {
        cudaGetLastError();
        g_mlp_err = "cudaMallocAsync failed";
        return OTGS_ENOMEM;
    }
    cudaMemcpyAsync(dtab, tab.data(), sizeof(FeatProb) * (size_t)nprob, cudaMemcpyHostToDevice, st);
    k_refine_src<<<(int)((M + 7) / 8), 256, 0, st>>>(dtab, nprob, M, alpha_hat, beta_hat, gamma, col0, in_dim, out);
    k_refine_tgt<<<(int)((N + 127) / 128), 128, 0, st>>>(dtab, nprob, M, N, alpha_hat, beta_hat, gamma, col0, in_dim,
                                                          out);
    cudaFreeAsync(dtab, st);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        g_mlp_err = std::string("second-pass features: ") + cudaGetErrorString(e);
        return OTGS_ECUDA;
    }
    return OTGS_OK;
}

}  // extern "C"
