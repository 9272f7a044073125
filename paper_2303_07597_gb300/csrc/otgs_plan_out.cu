// otgs_plan_out.cu -- downstream use of a solution: the transport plan and
// the barycentric mapping of the source samples.
//
// The plan at duals (alpha, beta) is the gradient of psi (Sec. 2.3, Eq. 5):
// t_ij = s_lj [alpha_i + beta_j - c_ij]_+ for row i of class l, with the
// block's shrink factor s_lj = [z - mu gamma]_+ / (gamma z), z the norm of
// the block's positive part.  The barycentric mapping (Sec. 2.1) moves the
// samples as n T^T X_S: target sample j's image is n sum_i t_ij x_i.
// Neither is on the solver's hot path: f is formed in FP64 here, once.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "otgs_handle.cuh"

namespace otgs {

namespace {

// s_lj for every (group, column): one thread per column, one grid row per
// group, the group's sorted rows walked in order (FP64).
__global__ void k_block_s(const float* __restrict__ C, int64_t ldc, const int32_t* __restrict__ goff,
                          const double* __restrict__ alpha_s, const double* __restrict__ beta, int n, double theta,
                          double gamma, double* s_out)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int l = blockIdx.y;
    if (j >= n) return;
    const int r0 = goff[l], r1 = goff[l + 1];
    double S = 0.0;
    const double bj = beta[j];
    for (int r = r0; r < r1; r++) {
        const double f = alpha_s[r] + bj - (double)C[(int64_t)r * ldc + j];
        if (f > 0.0) S += f * f;
    }
    const double z = sqrt(S);
    s_out[(int64_t)l * n + j] = z > theta ? (z - theta) / (gamma * z) : 0.0;
}

// t_ij into T (caller row order, row stride ldt), FP32.
__global__ void k_plan_dense(const float* __restrict__ C, int64_t ldc, const int32_t* __restrict__ perm,
                             const int32_t* __restrict__ rgroup, const double* __restrict__ alpha_s,
                             const double* __restrict__ beta, const double* __restrict__ s, int m, int n, float* T,
                             int64_t ldt)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (j >= n || r >= m) return;
    const double f = alpha_s[r] + beta[j] - (double)C[(int64_t)r * ldc + j];
    const double t = f > 0.0 ? s[(int64_t)rgroup[r] * n + j] * f : 0.0;
    T[(int64_t)perm[r] * ldt + j] = (float)t;
}

// out[j, c] = n sum_i T[i, j] X[i, c]: a 32 x 32 output tile per block of 256
// threads (4 outputs each), rows i in steps of 32 through shared memory, in
// order (deterministic), FP32 products added in FP32.
constexpr int BTILE = 32;
__global__ void __launch_bounds__(256) k_bary(const float* __restrict__ T, int64_t ldt, const float* __restrict__ X,
                                              int m, int n, int d, float scale, float* out)
{
    __shared__ float Ts[BTILE][BTILE + 1];  // [i][j]
    __shared__ float Xs[BTILE][BTILE + 1];  // [i][c]
    const int j0 = blockIdx.x * BTILE, c0 = blockIdx.y * BTILE;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // ty in [0, 8): rows ty, ty + 8, ...
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int i0 = 0; i0 < m; i0 += BTILE) {
        for (int q = ty; q < BTILE; q += 8) {
            const int i = i0 + q;
            Ts[q][tx] = (i < m && j0 + tx < n) ? T[(int64_t)i * ldt + j0 + tx] : 0.f;
            Xs[q][tx] = (i < m && c0 + tx < d) ? X[(int64_t)i * d + c0 + tx] : 0.f;
        }
        __syncthreads();
#pragma unroll 8
        for (int q = 0; q < BTILE; q++) {
            const float xv = Xs[q][tx];
#pragma unroll
            for (int u = 0; u < 4; u++) acc[u] = fmaf(Ts[q][ty + 8 * u], xv, acc[u]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; u++) {
        const int j = j0 + ty + 8 * u, c = c0 + tx;
        if (j < n && c < d) out[(int64_t)j * d + c] = scale * acc[u];
    }
}

// The plan of handle h at (alpha caller order, beta) into T (row stride ldt).
bool plan_into(Handle* h, const double* alpha, const double* beta, float* T, int64_t ldt)
{
    const ProbDesc& pd = h->probs_h[0];
    double* work = (double*)h->dalloc(sizeof(double) * ((size_t)h->m + (size_t)h->L * (size_t)h->n), "plan scratch");
    if (!work) return false;
    double* alpha_s = work;
    double* s = work + h->m;
    launch_permute_f64(alpha, h->dp.perm, (int32_t)h->m, alpha_s, true, h->st);
    const double theta = h->prm.mu * h->prm.gamma;
    dim3 g1((unsigned)((h->n + 127) / 128), (unsigned)h->L);
    k_block_s<<<g1, 128, 0, h->st>>>(pd.C, pd.ldc, h->dp.goff, alpha_s, beta, (int)h->n, theta, h->prm.gamma, s);
    for (int64_t r0 = 0; r0 < h->m; r0 += 65535) {
        const int rows = (int)std::min<int64_t>(65535, h->m - r0);
        dim3 g2((unsigned)((h->n + 127) / 128), (unsigned)rows);
        k_plan_dense<<<g2, 128, 0, h->st>>>(pd.C + r0 * pd.ldc, pd.ldc, h->dp.perm + r0, h->dp.rgroup + r0,
                                           alpha_s + r0, beta, s, rows, (int)h->n, T, ldt);
    }
    const bool ok = h->ck(cudaStreamSynchronize(h->st), "plan");
    for (size_t i = 0; i < h->allocs.size(); i++)
        if (h->allocs[i] == work) {
            h->allocs.erase(h->allocs.begin() + (long)i);
            break;
        }
    cudaFree(work);
    return ok && h->ck(cudaGetLastError(), "plan");
}

}  // namespace

}  // namespace otgs

using namespace otgs;

extern "C" {

int ot_gs_plan(ot_gs* hh, const double* alpha, const double* beta, float* T, int64_t ldt)
{
    if (!hh) return OTGS_EINVAL;
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!single_problem(h)) return OTGS_EINVAL;
    if (!alpha || !beta || !T || ldt < h->n) {
        h->fail(OTGS_EINVAL, "need alpha, beta, T and ldt >= n");
        return OTGS_EINVAL;
    }
    return plan_into(h, alpha, beta, T, ldt) ? OTGS_OK : h->last_code;
}

int ot_gs_barycentric(ot_gs* hh, const double* alpha, const double* beta, const float* XS, int32_t d, float* out)
{
    if (!hh) return OTGS_EINVAL;
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!single_problem(h)) return OTGS_EINVAL;
    if (!alpha || !beta || !XS || !out || d <= 0) {
        h->fail(OTGS_EINVAL, "need alpha, beta, XS, out and d > 0");
        return OTGS_EINVAL;
    }
    float* T = (float*)h->dalloc(sizeof(float) * (size_t)h->m * (size_t)h->n, "plan");
    if (!T) return h->last_code;
    bool ok = plan_into(h, alpha, beta, T, h->n);
    if (ok) {
        dim3 g((unsigned)((h->n + BTILE - 1) / BTILE), (unsigned)((d + BTILE - 1) / BTILE));
        k_bary<<<g, 256, 0, h->st>>>(T, h->n, XS, (int)h->m, (int)h->n, d, (float)h->n, out);
        ok = h->ck(cudaStreamSynchronize(h->st), "barycentric") && h->ck(cudaGetLastError(), "barycentric");
    }
    for (size_t i = 0; i < h->allocs.size(); i++)
        if (h->allocs[i] == T) {
            h->allocs.erase(h->allocs.begin() + (long)i);
            break;
        }
    cudaFree(T);
    return ok ? OTGS_OK : h->last_code;
}

}  // extern "C"
