// otgs_eval.cu -- the kernels around the evaluation of the dual (Eq. 4):
// the preparation of alpha and beta, the reduction of the evaluation
// kernel's sums into D and its gradient, and input utilities.
//
// Precision (the evaluation kernel is in otgs_stream.cu): near the optimum
// z - theta is tiny next to z, so z must be exact to ~1e-13 relative.  alpha
// and beta reach the kernel as FP32 (hi, lo) pairs plus an upper bound of each
// (bound_up) for the cheap bound and rejection tests; f is formed with
// error-free transformations where it may be positive.  Row and column sums
// of T and psi arrive as fixed-point integers, so results are deterministic
// whatever kernel formed a block and in whatever order, and screened
// evaluations (skipped units are exact zeros) equal dense ones bit for bit.
#include "otgs_internal.cuh"

namespace otgs {

#define FULLMASK 0xffffffffu

// --------------------------------------------------------------- prep
__global__ void k_prep(const double* __restrict__ alpha, int alpha_sorted, const int32_t* __restrict__ perm,
                       const double* __restrict__ beta, int m, int n, int npad, float4* rowA, float2* B2,
                       double* alpha_s_out, unsigned long long* rowfx, unsigned long long* colfx, EvalCtl* ctl)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    float apos = 0.f, bpos = 0.f;
    if (t < m) {
        const double a = alpha_sorted ? alpha[t] : alpha[perm[t]];
        apos = prep_row(a, rowA + t);
        rowfx[t] = 0ull;
        if (alpha_s_out) alpha_s_out[t] = a;
    }
    if (t < npad) {
        bpos = prep_col(t < n, t < n ? beta[t] : 0.0, B2 + t);
        if (t < n) colfx[t] = 0ull;
    }
    record_max(ctl, apos, bpos);
}

void launch_prep(const double* alpha, bool alpha_sorted, const int32_t* perm, const double* beta,
                 int32_t m, int32_t n, float4* rowA, float2* B2, double* alpha_s_out,
                 unsigned long long* rowfx, unsigned long long* colfx, EvalCtl* ctl, cudaStream_t st)
{
    const int npad = padded_cols(n);
    const int tot = m > npad ? m : npad;
    cudaMemsetAsync(ctl, 0, sizeof(EvalCtl), st);
    k_prep<<<(tot + 255) / 256, 256, 0, st>>>(alpha, alpha_sorted ? 1 : 0, perm, beta, m, n, npad, rowA, B2,
                                             alpha_s_out, rowfx, colfx, ctl);
}

// ------------------------------------------------------------- reduce
// One thread per sorted row and per column; the psi partials are split into
// one contiguous range per block.  Block sums meet in fixed trees and the
// last block to finish adds the block sums in block order, so the result does
// not depend on scheduling.
constexpr int RED_THREADS = 256;
constexpr int RED_WARPS = RED_THREADS / 32;
constexpr int BP = REDUCE_PARTS;  // values per block in block_part

int reduce_blocks(int32_t m, int32_t n)
{
    const int64_t tot = m > n ? m : n;
    return (int)((tot + RED_THREADS - 1) / RED_THREADS);
}

__global__ void __launch_bounds__(RED_THREADS) k_reduce(const ReduceArgs R)
{
    if (R.gate && !*R.gate) return;  // a skipped solver trial
    __shared__ double sh[3][RED_WARPS];
    __shared__ bool last;
    __shared__ FxScale fxs;  // once per block (FP64 scale arithmetic)
    if (threadIdx.x == 0) fxs = fx_scale(R.ctl->amax, R.ctl->bmax, R.fx_m, R.fx_n, R.gamma);
    __syncthreads();
    const FxScale& fx = fxs;
    const int t = blockIdx.x * RED_THREADS + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double ab = 0.0, dt = 0.0, inf = 0.0;
    if (t < R.m) {
        const double rs = (double)(long long)R.rowfx[t] * fx.from_r;
        const double ga = R.a_sorted[t] - rs;
        if (R.out_caller) R.out_caller[1 + R.perm[t]] = ga;
        if (R.G_sorted) R.G_sorted[t] = -ga;
        if (R.dir) dt = -ga * R.dir[t];
        inf = fabs(ga);
        ab = R.alpha_sorted[t] * R.a_sorted[t];
    }
    if (t < R.n) {
        const double cs = (double)(long long)R.colfx[t] * fx.from_c;
        const double gb = R.b[t] - cs;
        if (R.out_caller) R.out_caller[1 + R.m + t] = gb;
        if (R.G_sorted) R.G_sorted[R.m + t] = -gb;
        if (R.dir) dt += -gb * R.dir[R.m + t];
        inf = fmax(inf, fabs(gb));
        ab += R.beta[t] * R.b[t];
    }
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        ab += __shfl_xor_sync(FULLMASK, ab, off);
        dt += __shfl_xor_sync(FULLMASK, dt, off);
        inf = fmax(inf, __shfl_xor_sync(FULLMASK, inf, off));
    }
    if (lane == 0) {
        sh[0][warp] = ab;
        sh[1][warp] = dt;
        sh[2][warp] = inf;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double v0 = 0.0, v1 = 0.0, v2 = 0.0;
        for (int w = 0; w < RED_WARPS; w++) {
            v0 += sh[0][w];
            v1 += sh[1][w];
            v2 = fmax(v2, sh[2][w]);
        }
        R.block_part[BP * blockIdx.x + 0] = v0;
        R.block_part[BP * blockIdx.x + 1] = v1;
        R.block_part[BP * blockIdx.x + 2] = v2;
        __threadfence();
        const unsigned ticket = atomicAdd(R.counter, 1u);
        last = ticket == gridDim.x - 1;
    }
    __syncthreads();
    if (!last || threadIdx.x >= 32) return;
    __threadfence();
    // last block, first warp: fixed-order sums over blocks
    const volatile double* bp = R.block_part;
    double s_ab = 0.0, s_dt = 0.0, s_inf = 0.0;
    for (int b = lane; b < (int)gridDim.x; b += 32) {
        s_ab += bp[BP * b];
        s_dt += bp[BP * b + 1];
        s_inf = fmax(s_inf, bp[BP * b + 2]);
    }
    for (int off = 16; off >= 1; off >>= 1) {
        s_ab += __shfl_xor_sync(FULLMASK, s_ab, off);
        s_dt += __shfl_xor_sync(FULLMASK, s_dt, off);
        s_inf = fmax(s_inf, __shfl_xor_sync(FULLMASK, s_inf, off));
    }
    if (lane == 0) {
        // psi: the exact-sum kernel's fixed-point sums
        const double s_psi = psi_from_fx((long long)R.psix[0], (long long)R.psix[1], fx.from_p);
        const double D = (R.err && *(volatile const int*)R.err) ? __longlong_as_double(0x7ff8000000000000ll)
                                                                  : s_ab - s_psi;
        if (R.out_caller) R.out_caller[0] = D;
        if (R.scal) {
            R.scal[0] = D;
            R.scal[1] = s_dt;
            R.scal[2] = s_inf;
            R.scal[3] = s_psi;
        }
        *R.counter = 0u;
    }
}

void launch_reduce(const ReduceArgs& a, cudaStream_t st)
{
    k_reduce<<<reduce_blocks(a.m, a.n), RED_THREADS, 0, st>>>(a);
}

// ---------------------------------------------------------- utilities
__global__ void k_gather_rows(const float* __restrict__ C, int64_t ldc, const int32_t* __restrict__ perm,
                              int32_t base, int32_t m, int32_t n, float* Cs, int64_t ldcs)
{
    const int r = blockIdx.y;
    const float* src = C + (int64_t)(perm[r] - base) * ldc;
    float* dst = Cs + (int64_t)r * ldcs;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < ldcs; j += (int64_t)gridDim.x * blockDim.x)
        dst[j] = j < n ? src[j] : 0.f;
}

void launch_gather_rows(const float* C, int64_t ldc, const int32_t* perm, int32_t base, int32_t m, int32_t n,
                        float* Cs, int64_t ldcs, cudaStream_t st)
{
    int bx = (int)((ldcs + 255) / 256);
    if (bx > 64) bx = 64;
    for (int32_t r0 = 0; r0 < m; r0 += 65535) {
        int32_t rows = m - r0 < 65535 ? m - r0 : 65535;
        dim3 grid(bx, rows);
        k_gather_rows<<<grid, 256, 0, st>>>(C, ldc, perm + r0, base, rows, n, Cs + (int64_t)r0 * ldcs, ldcs);
    }
}

// CT[j * ldct + i] = C[i * ldc + j], i < m, j < n: 32 x 32 tiles through shared
// memory (reads along C's rows, writes along CT's rows, both coalesced).
__global__ void __launch_bounds__(256) k_transpose(const float* __restrict__ C, int64_t ldc, int32_t m, int32_t n,
                                                   float* __restrict__ CT, int64_t ldct)
{
    __shared__ float t[32][33];
    const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int r = ty; r < 32; r += 8) {
        const int i = i0 + r, j = j0 + tx;
        t[r][tx] = (i < m && j < n) ? C[(int64_t)i * ldc + j] : 0.f;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int j = j0 + r, i = i0 + tx;
        if (j < n && i < m) CT[(int64_t)j * ldct + i] = t[tx][r];
    }
}

void launch_transpose(const float* C, int64_t ldc, int32_t m, int32_t n, float* CT, int64_t ldct, cudaStream_t st)
{
    for (int32_t i0 = 0; i0 < m; i0 += 32 * 65535) {
        const int32_t rows = m - i0 < 32 * 65535 ? m - i0 : 32 * 65535;
        dim3 grid((unsigned)((n + 31) / 32), (unsigned)((rows + 31) / 32));
        k_transpose<<<grid, 256, 0, st>>>(C + (int64_t)i0 * ldc, ldc, rows, n, CT + i0, ldct);
    }
}

__global__ void k_permute(const double* __restrict__ src, const int32_t* __restrict__ perm, int32_t m,
                          double* dst, int to_sorted)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= m) return;
    if (to_sorted) dst[r] = src[perm[r]];
    else dst[perm[r]] = src[r];
}

void launch_permute_f64(const double* src, const int32_t* perm, int32_t m, double* dst, bool to_sorted,
                        cudaStream_t st)
{
    k_permute<<<(m + 255) / 256, 256, 0, st>>>(src, perm, m, dst, to_sorted ? 1 : 0);
}

// flags[0]: C has a non-finite entry; flags[1]: C has a negative entry;
// flags[2]: a or b has a non-positive or non-finite entry; flags[3]: bits of max c.
// sums[0..1] = sum a, sum b.
__global__ void k_check(const float* __restrict__ C, int64_t ldc, int32_t m, int32_t n,
                        const double* __restrict__ a, const double* __restrict__ b, double* sums, int* flags)
{
    int bad_f = 0, bad_n = 0, bad_m = 0;
    const int64_t tot = (int64_t)m * n;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < tot; k += (int64_t)gridDim.x * blockDim.x) {
        float c = C[(k / n) * ldc + (k % n)];
        if (!isfinite(c)) bad_f = 1;
        else if (c < 0.f) bad_n = 1;
    }
    double sa = 0.0, sb = 0.0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x) {
        double v = a[k];
        if (!(v > 0.0) || !isfinite(v)) bad_m = 1;
        sa += v;
    }
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        double v = b[k];
        if (!(v > 0.0) || !isfinite(v)) bad_m = 1;
        sb += v;
    }
    float cm = 0.f;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < tot; k += (int64_t)gridDim.x * blockDim.x) {
        float c = C[(k / n) * ldc + (k % n)];
        if (c > cm) cm = c;  // NaN compares false
    }
    for (int off = 16; off >= 1; off >>= 1) cm = fmaxf(cm, __shfl_xor_sync(FULLMASK, cm, off));
    if ((threadIdx.x & 31) == 0) atomicMax((unsigned*)(flags + 3), __float_as_uint(cm));
    if (__any_sync(FULLMASK, bad_f) && (threadIdx.x & 31) == 0) atomicOr(flags + 0, 1);
    if (__any_sync(FULLMASK, bad_n) && (threadIdx.x & 31) == 0) atomicOr(flags + 1, 1);
    if (__any_sync(FULLMASK, bad_m) && (threadIdx.x & 31) == 0) atomicOr(flags + 2, 1);
    atomicAdd(sums + 0, sa);
    atomicAdd(sums + 1, sb);
}

void launch_check_finite(const float* C, int64_t ldc, int32_t m, int32_t n, const double* a, const double* b,
                         double* sums, int* flags, cudaStream_t st)
{
    k_check<<<1024, 256, 0, st>>>(C, ldc, m, n, a, b, sums, flags);
}

}  // namespace otgs
