// otgs_eval.cu -- evaluation of the smooth dual (Eq. 4) and its gradient.
//
// One pass streams C once.  For every unit (group l, 32-column tile) the
// kernel forms f = alpha_i + beta_j - c_ij, the positive part p = [f]_+,
// S = ||p||^2 and P = sum p per column, then the group soft-threshold of
// Eq. 5: z = sqrt(S), s = [z - theta]_+ / (gamma z), psi = [z - theta]_+^2/(2 gamma).
// Row sums s p_ij (second pass over the unit, from L1/L2), column sums s P and
// psi go to per-item partial buffers that the reduction kernel adds in a
// fixed order, so results are deterministic and identical whether or not
// units were skipped by screening (skipped units are exact zeros).
//
// Precision: near the optimum z - theta is tiny next to z, so z must be exact
// to ~1e-13 relative.  alpha and beta arrive as FP32 (hi, lo) pairs; a cheap
// FP32 test rejects elements whose f is certainly <= 0, and for the rest f is
// formed with error-free transformations (TwoSum) as a float pair, squared and
// summed in double-float.  FP64 is used only per block for psi.
#include "otgs_internal.cuh"

namespace otgs {

#define FULLMASK 0xffffffffu

// Knuth's TwoSum: s + e == a + b exactly (round-to-nearest).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (h, l) += (oh, ol); symmetric in its arguments bit for bit.
__device__ __forceinline__ void df_add(float& h, float& l, float oh, float ol)
{
    float s, e;
    two_sum(h, oh, s, e);
    h = s;
    l = __fadd_rn(__fadd_rn(l, ol), e);
}

// f = (ah + al) + (bh + bl) - c as a float pair (fh, fl), |error| ~ 2^-46 (|alpha|+|beta|+c).
__device__ __forceinline__ void f_exact(float ah, float al, float bh, float bl, float c,
                                        float& fh, float& fl)
{
    float s1, e1, s2, e2;
    two_sum(ah, -c, s1, e1);
    two_sum(s1, bh, s2, e2);
    float t = __fadd_rn(__fadd_rn(e1, e2), __fadd_rn(al, bl));
    fh = __fadd_rn(s2, t);
    fl = __fsub_rn(t, __fsub_rn(fh, s2));
}

// S += p^2 and P += p in double-float for p = (fh, fl) > 0.
__device__ __forceinline__ void acc_p(float fh, float fl, float& Sh, float& Sl, float& Ph, float& Pl)
{
    float q = __fmul_rn(fh, fh);
    float ql = fmaf(fh, fh, -q);
    ql = fmaf(2.f * fh, fl, ql);
    df_add(Sh, Sl, q, ql);
    df_add(Ph, Pl, fh, fl);
}

// Eq. 5 for one block from S = ||[f_[l]]_+||^2: returns the shrink factor
// s = [z - theta]_+ / (gamma z) and psi = [z - theta]_+^2 / (2 gamma).
__device__ __forceinline__ float block_scale(float Sh, float Sl, const EvalArgs& A, double& psi)
{
    psi = 0.0;
    if (!(Sh > 0.f) || Sh < A.th2_cut) return 0.f;
    float sh = __fadd_rn(Sh, Sl);
    float sl = __fsub_rn(Sl, __fsub_rn(sh, Sh));
    float zh = __fsqrt_rn(sh);
    float res = __fadd_rn(fmaf(-zh, zh, sh), sl);
    float zl = __fdiv_rn(res, __fmul_rn(2.f, zh));
    float dh, de;
    two_sum(zh, -A.theta_hi, dh, de);
    float dl = __fadd_rn(de, __fsub_rn(zl, A.theta_lo));
    float ds = __fadd_rn(dh, dl);
    if (!(ds > 0.f)) return 0.f;
    double d = (double)dh + (double)dl;
    psi = d * d * A.inv2g;
    return __fdiv_rn(ds, __fmul_rn(A.gamma, __fadd_rn(zh, zl)));
}

// z rounded up (snapshot value z~ of Def. 1, kept as an upper bound).
__device__ __forceinline__ float z_up(float Sh, float Sl)
{
    return __fsqrt_ru(fmaxf(__fadd_ru(Sh, Sl), 0.f));
}

__device__ __forceinline__ float4 ld_c4(const float* p, bool ok)
{
    return ok ? __ldg(reinterpret_cast<const float4*>(p)) : make_float4(3e38f, 3e38f, 3e38f, 3e38f);
}

__device__ __forceinline__ bool unit_bit(const uint32_t* need, int words, int l, int jt)
{
    return (__ldg(need + (int64_t)l * words + (jt >> 5)) >> (jt & 31)) & 1u;
}

// Pass A over the rows assigned to this lane (row = r0 + first + k*step):
// accumulates S, P (double-float) and, for snapshots, O = ||[f]_-||^2 (FP32).
template <bool SNAP>
__device__ __forceinline__ bool pass_a(const EvalArgs& A, int r0, int first, int step, int g,
                                       int col, bool cv, const float bh[4], const float bl[4],
                                       const float sb[4], float Sh[4], float Sl[4], float Ph[4],
                                       float Pl[4], float O[4])
{
    bool anyc = false;
    const float* cp = A.C + (int64_t)r0 * A.ldc + col;
    int r = first;
    for (; r + 3 * step < g; r += 4 * step) {
        float4 c4[4];
        float2 a2[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            c4[u] = ld_c4(cp + (int64_t)(r + u * step) * A.ldc, cv);
            a2[u] = __ldg(A.A2 + r0 + r + u * step);
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const float c[4] = {c4[u].x, c4[u].y, c4[u].z, c4[u].w};
            const float sa = fabsf(a2[u].x) * 0x1p-22f;
#pragma unroll
            for (int k = 0; k < 4; k++) {
                float x = __fsub_rn(__fadd_rn(a2[u].x, bh[k]), c[k]);
                if (SNAP) { float mn = fminf(x, 0.f); O[k] = fmaf(mn, mn, O[k]); }
                if (__fadd_rn(x, __fadd_rn(sa, sb[k])) > 0.f) {
                    float fh, fl;
                    f_exact(a2[u].x, a2[u].y, bh[k], bl[k], c[k], fh, fl);
                    if (fh > 0.f) { acc_p(fh, fl, Sh[k], Sl[k], Ph[k], Pl[k]); anyc = true; }
                }
            }
        }
    }
    for (; r < g; r += step) {
        float4 c4 = ld_c4(cp + (int64_t)r * A.ldc, cv);
        float2 a2 = __ldg(A.A2 + r0 + r);
        const float c[4] = {c4.x, c4.y, c4.z, c4.w};
        const float sa = fabsf(a2.x) * 0x1p-22f;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            float x = __fsub_rn(__fadd_rn(a2.x, bh[k]), c[k]);
            if (SNAP) { float mn = fminf(x, 0.f); O[k] = fmaf(mn, mn, O[k]); }
            if (__fadd_rn(x, __fadd_rn(sa, sb[k])) > 0.f) {
                float fh, fl;
                f_exact(a2.x, a2.y, bh[k], bl[k], c[k], fh, fl);
                if (fh > 0.f) { acc_p(fh, fl, Sh[k], Sl[k], Ph[k], Pl[k]); anyc = true; }
            }
        }
    }
    return anyc;
}

// Row sum of s_k p_ij over this lane's 4 columns for one row.
__device__ __forceinline__ float row_part(const EvalArgs& A, float2 a2, float4 c4, const float bh[4],
                                          const float bl[4], const float sb[4], const float s[4])
{
    const float c[4] = {c4.x, c4.y, c4.z, c4.w};
    const float sa = fabsf(a2.x) * 0x1p-22f;
    float rs = 0.f;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        if (s[k] > 0.f) {
            float x = __fsub_rn(__fadd_rn(a2.x, bh[k]), c[k]);
            if (__fadd_rn(x, __fadd_rn(sa, sb[k])) > 0.f) {
                float fh, fl;
                f_exact(a2.x, a2.y, bh[k], bl[k], c[k], fh, fl);
                if (fh > 0.f) rs = fmaf(s[k], fh, rs);
            }
        }
    }
    return rs;
}

// Pass B: row sums into racc[r] for this lane's rows; lanes of one row-slot
// (8 lanes, mask smask) reduce their 32 columns with a fixed xor tree.
__device__ __forceinline__ void pass_b(const EvalArgs& A, int r0, int first, int step, int g, int col,
                                       bool cv, const float bh[4], const float bl[4],
                                       const float sb[4], const float s[4], double* racc, int q,
                                       unsigned smask)
{
    const float* cp = A.C + (int64_t)r0 * A.ldc + col;
    int r = first;
    for (; r + step < g; r += 2 * step) {
        float4 c0 = ld_c4(cp + (int64_t)r * A.ldc, cv);
        float4 c1 = ld_c4(cp + (int64_t)(r + step) * A.ldc, cv);
        float2 a0 = __ldg(A.A2 + r0 + r), a1 = __ldg(A.A2 + r0 + r + step);
        float rs0 = row_part(A, a0, c0, bh, bl, sb, s);
        float rs1 = row_part(A, a1, c1, bh, bl, sb, s);
        rs0 += __shfl_xor_sync(smask, rs0, 1);
        rs1 += __shfl_xor_sync(smask, rs1, 1);
        rs0 += __shfl_xor_sync(smask, rs0, 2);
        rs1 += __shfl_xor_sync(smask, rs1, 2);
        rs0 += __shfl_xor_sync(smask, rs0, 4);
        rs1 += __shfl_xor_sync(smask, rs1, 4);
        if (q == 0) {
            racc[r] += (double)rs0;
            racc[r + step] += (double)rs1;
        }
    }
    for (; r < g; r += step) {
        float4 c0 = ld_c4(cp + (int64_t)r * A.ldc, cv);
        float2 a0 = __ldg(A.A2 + r0 + r);
        float rs0 = row_part(A, a0, c0, bh, bl, sb, s);
        rs0 += __shfl_xor_sync(smask, rs0, 1);
        rs0 += __shfl_xor_sync(smask, rs0, 2);
        rs0 += __shfl_xor_sync(smask, rs0, 4);
        if (q == 0) racc[r] += (double)rs0;
    }
}

__device__ __forceinline__ void load_cols(const EvalArgs& A, int col, float bh[4], float bl[4], float sb[4])
{
    const float4* b4 = reinterpret_cast<const float4*>(A.B2 + col);
    float4 u = __ldg(b4), v = __ldg(b4 + 1);
    bh[0] = u.x; bl[0] = u.y; bh[1] = u.z; bl[1] = u.w;
    bh[2] = v.x; bl[2] = v.y; bh[3] = v.z; bl[3] = v.w;
#pragma unroll
    for (int k = 0; k < 4; k++) sb[k] = fabsf(bh[k]) * 0x1p-22f;
}

__device__ __forceinline__ void write_snap(const EvalArgs& A, int l, int col, const float zt[4],
                                           const float ot[4])
{
    const int64_t ldz = (int64_t)A.ntiles * TW;
    float4 z4, o4;
    z4.x = col + 0 < A.n ? zt[0] : 0.f; o4.x = col + 0 < A.n ? ot[0] : 0.f;
    z4.y = col + 1 < A.n ? zt[1] : 0.f; o4.y = col + 1 < A.n ? ot[1] : 0.f;
    z4.z = col + 2 < A.n ? zt[2] : 0.f; o4.z = col + 2 < A.n ? ot[2] : 0.f;
    z4.w = col + 3 < A.n ? zt[3] : 0.f; o4.w = col + 3 < A.n ? ot[3] : 0.f;
    reinterpret_cast<float4*>(A.zt + (int64_t)l * ldz + col)[0] = z4;
    reinterpret_cast<float4*>(A.ot + (int64_t)l * ldz + col)[0] = o4;
}

// One unit processed by one warp (small panels).
template <bool SNAP>
__device__ __forceinline__ void unit_small(const EvalArgs& A, int l, int jt, double* racc,
                                           double cacc[4], double& psi_acc)
{
    const int lane = threadIdx.x & 31, slot = lane >> 3, q = lane & 7;
    const int r0 = A.plan.goff[l];
    const int g = A.plan.goff[l + 1] - r0;
    const int col = jt * TW + q * 4;
    const bool cv = col < A.n;
    float bh[4], bl[4], sb[4];
    load_cols(A, col, bh, bl, sb);
    float Sh[4] = {0, 0, 0, 0}, Sl[4] = {0, 0, 0, 0}, Ph[4] = {0, 0, 0, 0}, Pl[4] = {0, 0, 0, 0};
    float O[4] = {0, 0, 0, 0};
    bool anyc = pass_a<SNAP>(A, r0, slot, 4, g, col, cv, bh, bl, sb, Sh, Sl, Ph, Pl, O);
    if (SNAP) {
#pragma unroll
        for (int k = 0; k < 4; k++) {
            O[k] += __shfl_xor_sync(FULLMASK, O[k], 8);
            O[k] += __shfl_xor_sync(FULLMASK, O[k], 16);
        }
    }
    if (!__any_sync(FULLMASK, anyc)) {
        if (SNAP && slot == 0) {
            float zt[4] = {0, 0, 0, 0}, ot[4];
#pragma unroll
            for (int k = 0; k < 4; k++) ot[k] = __fsqrt_ru(O[k]);
            write_snap(A, l, col, zt, ot);
        }
        return;
    }
#pragma unroll
    for (int k = 0; k < 4; k++) {
#pragma unroll
        for (int off = 8; off <= 16; off <<= 1) {
            float a = __shfl_xor_sync(FULLMASK, Sh[k], off), b = __shfl_xor_sync(FULLMASK, Sl[k], off);
            float c = __shfl_xor_sync(FULLMASK, Ph[k], off), d = __shfl_xor_sync(FULLMASK, Pl[k], off);
            df_add(Sh[k], Sl[k], a, b);
            df_add(Ph[k], Pl[k], c, d);
        }
    }
    float s[4];
    bool anyact = false;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        double psi;
        s[k] = block_scale(Sh[k], Sl[k], A, psi);
        if (slot == 0) psi_acc += psi;
        anyact |= s[k] > 0.f;
    }
    if (SNAP && slot == 0) {
        float zt[4], ot[4];
#pragma unroll
        for (int k = 0; k < 4; k++) { zt[k] = z_up(Sh[k], Sl[k]); ot[k] = __fsqrt_ru(O[k]); }
        write_snap(A, l, col, zt, ot);
    }
    if (!__any_sync(FULLMASK, anyact)) return;
    if (slot == 0) {
#pragma unroll
        for (int k = 0; k < 4; k++) cacc[k] += (double)__fmul_rn(s[k], __fadd_rn(Ph[k], Pl[k]));
    }
    pass_b(A, r0, slot, 4, g, col, cv, bh, bl, sb, s, racc, q, 0xffu << (slot * 8));
}

template <bool SNAP>
__device__ void small_item(const EvalArgs& A, int item, int p, int cc, double* smem)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, slot = lane >> 3, q = lane & 7;
    const int W = A.plan.pW[p], rows = A.plan.prows[p];
    const int col0 = cc * W;
    const int ncols = min(W, A.n - col0);
    const int nt = (ncols + TW - 1) / TW, t0 = col0 / TW;
    double* racc = smem;                   // [PANEL_ROWS]
    double* colacc = smem + PANEL_ROWS;    // [NWARPS][SMALL_CHUNK]
    __shared__ double psi_w[NWARPS];
    for (int i = threadIdx.x; i < rows; i += NTHREADS) racc[i] = 0.0;
    __syncthreads();
    const int gb = A.plan.pw_off[p * NWARPS + warp], ge = A.plan.pw_off[p * NWARPS + warp + 1];
    double psi_acc = 0.0;
    for (int t = 0; t < nt; t++) {
        const int jt = t0 + t;
        double cacc[4] = {0.0, 0.0, 0.0, 0.0};
        for (int gi = gb; gi < ge; gi++) {
            const int l = A.plan.pgrp[gi];
            if (A.unit_need && !unit_bit(A.unit_need, A.unit_words, l, jt)) continue;
            unit_small<SNAP>(A, l, jt, racc + A.plan.gsrow[l], cacc, psi_acc);
        }
        if (slot == 0) {
            double* dst = colacc + warp * SMALL_CHUNK + t * TW + q * 4;
            dst[0] = cacc[0]; dst[1] = cacc[1]; dst[2] = cacc[2]; dst[3] = cacc[3];
        }
    }
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) psi_acc += __shfl_xor_sync(FULLMASK, psi_acc, off);
    if (lane == 0) psi_w[warp] = psi_acc;
    __syncthreads();
    const int64_t rbase = A.plan.prp[p] + (int64_t)cc * rows;
    for (int i = threadIdx.x; i < rows; i += NTHREADS) A.rowpart[rbase + i] = racc[i];
    for (int c = threadIdx.x; c < ncols; c += NTHREADS) {
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < NWARPS; w++) s += colacc[w * SMALL_CHUNK + c];
        A.colpart[(int64_t)p * A.n + col0 + c] = s;
    }
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < NWARPS; w++) s += psi_w[w];
        A.psipart[item] = s;
    }
}

// One big group: the CTA's 32 row-slots (8 warps x 4) split its rows; the
// per-column partials meet in shared memory and are combined in warp order.
template <bool SNAP>
__device__ void big_item(const EvalArgs& A, int item, int p, int cc, double* smem)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, slot = lane >> 3, q = lane & 7;
    const int l = A.plan.pgrp[A.plan.pw_off[p * NWARPS]];
    const int r0 = A.plan.goff[l], g = A.plan.goff[l + 1] - r0;
    const int W = A.plan.pW[p];
    const int col0 = cc * W;
    const int ncols = min(W, A.n - col0);
    const int nt = (ncols + TW - 1) / TW, t0 = col0 / TW;
    const int64_t rbase = A.plan.prp[p] + (int64_t)cc * g;
    const bool in_smem = g <= BIG_SMEM_ROWS;
    double* racc = in_smem ? smem : A.rowpart + rbase;
    float4* red = reinterpret_cast<float4*>(smem + BIG_SMEM_ROWS);     // [2][NWARPS][TW]
    float* redO = reinterpret_cast<float*>(red + 2 * NWARPS * TW);      // [2][NWARPS][TW]
    const int first = warp * 4 + slot;   // this lane's first row; step 32
    const int step = NWARPS * 4;
    if (q == 0)
        for (int r = first; r < g; r += step) racc[r] = 0.0;
    double psi_acc = 0.0;
    int nproc = 0;  // processed units; the partial buffers alternate per processed unit
    for (int t = 0; t < nt; t++) {
        const int jt = t0 + t;
        const int col = jt * TW + q * 4;
        const bool cv = col < A.n;
        if (A.unit_need && !unit_bit(A.unit_need, A.unit_words, l, jt)) {
            if (warp == 0 && slot == 0)
                for (int k = 0; k < 4; k++)
                    if (col + k < A.n) A.colpart[(int64_t)p * A.n + col + k] = 0.0;
            continue;
        }
        const int buf = nproc & 1;
        nproc++;
        float bh[4], bl[4], sb[4];
        load_cols(A, col, bh, bl, sb);
        float Sh[4] = {0, 0, 0, 0}, Sl[4] = {0, 0, 0, 0}, Ph[4] = {0, 0, 0, 0}, Pl[4] = {0, 0, 0, 0};
        float O[4] = {0, 0, 0, 0};
        bool anyc = pass_a<SNAP>(A, r0, first, step, g, col, cv, bh, bl, sb, Sh, Sl, Ph, Pl, O);
#pragma unroll
        for (int k = 0; k < 4; k++) {
#pragma unroll
            for (int off = 8; off <= 16; off <<= 1) {
                float a = __shfl_xor_sync(FULLMASK, Sh[k], off), b = __shfl_xor_sync(FULLMASK, Sl[k], off);
                float c = __shfl_xor_sync(FULLMASK, Ph[k], off), d = __shfl_xor_sync(FULLMASK, Pl[k], off);
                df_add(Sh[k], Sl[k], a, b);
                df_add(Ph[k], Pl[k], c, d);
                if (SNAP) O[k] += __shfl_xor_sync(FULLMASK, O[k], off);
            }
        }
        if (slot == 0) {
#pragma unroll
            for (int k = 0; k < 4; k++) {
                red[(buf * NWARPS + warp) * TW + q * 4 + k] = make_float4(Sh[k], Sl[k], Ph[k], Pl[k]);
                if (SNAP) redO[(buf * NWARPS + warp) * TW + q * 4 + k] = O[k];
            }
        }
        const int any = __syncthreads_or(anyc ? 1 : 0);
        // every warp combines the NWARPS partials in the same order
        float s[4] = {0, 0, 0, 0};
        float zt[4] = {0, 0, 0, 0}, ot[4] = {0, 0, 0, 0};
        bool anyact = false;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const int c = q * 4 + k;
            if (SNAP) {
                float o = redO[(buf * NWARPS) * TW + c];
                for (int w = 1; w < NWARPS; w++) o += redO[(buf * NWARPS + w) * TW + c];
                ot[k] = __fsqrt_ru(o);
            }
            if (!any) continue;
            float4 v = red[(buf * NWARPS) * TW + c];
            float h = v.x, lo = v.y, ph = v.z, pl = v.w;
            for (int w = 1; w < NWARPS; w++) {
                float4 u = red[(buf * NWARPS + w) * TW + c];
                df_add(h, lo, u.x, u.y);
                df_add(ph, pl, u.z, u.w);
            }
            double psi;
            s[k] = block_scale(h, lo, A, psi);
            if (warp == 0 && slot == 0) psi_acc += psi;
            anyact |= s[k] > 0.f;
            zt[k] = z_up(h, lo);
            if (warp == 0 && slot == 0 && col + k < A.n)
                A.colpart[(int64_t)p * A.n + col + k] = (double)__fmul_rn(s[k], __fadd_rn(ph, pl));
        }
        if (!any && warp == 0 && slot == 0)
            for (int k = 0; k < 4; k++)
                if (col + k < A.n) A.colpart[(int64_t)p * A.n + col + k] = 0.0;
        if (SNAP && warp == 0 && slot == 0) write_snap(A, l, col, zt, ot);
        if (__any_sync(FULLMASK, anyact))
            pass_b(A, r0, first, step, g, col, cv, bh, bl, sb, s, racc, q, 0xffu << (slot * 8));
    }
    __shared__ double psi_b;
    if (warp == 0) {
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) psi_acc += __shfl_xor_sync(FULLMASK, psi_acc, off);
        if (lane == 0) psi_b = psi_acc;
    }
    __syncthreads();
    if (in_smem)
        for (int i = threadIdx.x; i < g; i += NTHREADS) A.rowpart[rbase + i] = racc[i];
    if (threadIdx.x == 0) A.psipart[item] = psi_b;
}

template <bool SNAP>
__global__ void __launch_bounds__(NTHREADS, 2) k_eval(const EvalArgs A)
{
    extern __shared__ double smem[];
    const int item = A.items[blockIdx.x];
    if (A.unit_need && !A.item_active[item]) return;  // screened: nothing to stream
    const int p = A.plan.item_panel[item], cc = A.plan.item_chunk[item];
    if (A.plan.pkind[p] == 0) small_item<SNAP>(A, item, p, cc, smem);
    else big_item<SNAP>(A, item, p, cc, smem);
}

size_t eval_smem_bytes()
{
    size_t small = sizeof(double) * (PANEL_ROWS + NWARPS * SMALL_CHUNK);
    size_t big = sizeof(double) * BIG_SMEM_ROWS + 2 * NWARPS * TW * (sizeof(float4) + sizeof(float));
    return small > big ? small : big;
}

void launch_eval(const EvalArgs& a, int n_ctas, cudaStream_t st)
{
    if (n_ctas <= 0) return;
    size_t sm = eval_smem_bytes();
    if (a.zt) k_eval<true><<<n_ctas, NTHREADS, sm, st>>>(a);
    else k_eval<false><<<n_ctas, NTHREADS, sm, st>>>(a);
}

// --------------------------------------------------------------- prep
__device__ __forceinline__ float2 split2(double x)
{
    float h = __double2float_rn(x);
    return make_float2(h, __double2float_rn(x - (double)h));
}

__global__ void k_prep(const double* __restrict__ alpha, int alpha_sorted, const int32_t* __restrict__ perm,
                       const double* __restrict__ beta, int m, int n, int npad, float2* A2, float2* B2,
                       double* alpha_s_out)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < m) {
        double a = alpha_sorted ? alpha[t] : alpha[perm[t]];
        A2[t] = split2(a);
        if (alpha_s_out) alpha_s_out[t] = a;
    }
    if (t < npad) B2[t] = t < n ? split2(beta[t]) : make_float2(-1e30f, 0.f);
}

void launch_prep(const double* alpha, bool alpha_sorted, const int32_t* perm, const double* beta,
                 int32_t m, int32_t n, int32_t ntiles, float2* A2, float2* B2, double* alpha_s_out,
                 cudaStream_t st)
{
    int npad = ntiles * TW;
    int tot = m > npad ? m : npad;
    k_prep<<<(tot + 255) / 256, 256, 0, st>>>(alpha, alpha_sorted ? 1 : 0, perm, beta, m, n, npad, A2, B2,
                                             alpha_s_out);
}

// ------------------------------------------------------------- reduce
// Eight lanes per row and per column: lane k adds the partials k, k+8, ...
// and the eight lane sums meet in a fixed xor tree, so the result does not
// depend on scheduling.
constexpr int RED_THREADS = 256;
constexpr int RED_LANES = 8;

int reduce_blocks(int32_t m, int32_t n)
{
    int64_t tot = (int64_t)(m > n ? m : n) * RED_LANES;
    return (int)((tot + RED_THREADS - 1) / RED_THREADS);
}

__global__ void __launch_bounds__(RED_THREADS) k_reduce(const ReduceArgs R)
{
    __shared__ double sh[3][RED_THREADS / RED_LANES];
    __shared__ bool last;
    const int gt = blockIdx.x * RED_THREADS + threadIdx.x;
    const int t = gt / RED_LANES, k = gt % RED_LANES;
    const unsigned gmask = 0xffu << (threadIdx.x & 24);
    double ab = 0.0, dt = 0.0, inf = 0.0;
    if (t < R.m) {
        const int l = R.plan.rgroup[t];
        const int p = R.plan.gpanel[l];
        const int loc = R.plan.gsrow[l] + (t - R.plan.goff[l]);
        const int rows = R.plan.prows[p], nch = R.plan.pnch[p], it0 = R.plan.pitem[p];
        const double* rp = R.rowpart + R.plan.prp[p] + loc;
        double acc = 0.0;
#pragma unroll 4
        for (int c = k; c < nch; c += RED_LANES) {
            const double v = __ldg(rp + (int64_t)c * rows);
            acc += __ldg(R.item_active + it0 + c) ? v : 0.0;
        }
        acc += __shfl_xor_sync(gmask, acc, 1);
        acc += __shfl_xor_sync(gmask, acc, 2);
        acc += __shfl_xor_sync(gmask, acc, 4);
        const double ga = R.a_sorted[t] - acc;
        if (k == 0) {
            if (R.out_caller) R.out_caller[1 + R.plan.perm[t]] = ga;
            if (R.G_sorted) R.G_sorted[t] = -ga;
            if (R.dir) dt = -ga * R.dir[t];
            inf = fabs(ga);
            ab = R.alpha_sorted[t] * R.a_sorted[t];
        }
    }
    if (t < R.n) {
        double acc = 0.0;
#pragma unroll 4
        for (int p = k; p < R.npanels; p += RED_LANES) {
            const int c = t / __ldg(R.plan.pW + p);
            const double v = __ldg(R.colpart + (int64_t)p * R.n + t);
            acc += __ldg(R.item_active + __ldg(R.plan.pitem + p) + c) ? v : 0.0;
        }
        acc += __shfl_xor_sync(gmask, acc, 1);
        acc += __shfl_xor_sync(gmask, acc, 2);
        acc += __shfl_xor_sync(gmask, acc, 4);
        const double gb = R.b[t] - acc;
        if (k == 0) {
            if (R.out_caller) R.out_caller[1 + R.m + t] = gb;
            if (R.G_sorted) R.G_sorted[R.m + t] = -gb;
            if (R.dir) dt += -gb * R.dir[R.m + t];
            inf = fmax(inf, fabs(gb));
            ab += R.beta[t] * R.b[t];
        }
    }
    const int g = threadIdx.x / RED_LANES;
    if (k == 0) {
        sh[0][g] = ab;
        sh[1][g] = dt;
        sh[2][g] = inf;
    }
    __syncthreads();
    for (int s = RED_THREADS / RED_LANES / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + s];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + s];
            sh[2][threadIdx.x] = fmax(sh[2][threadIdx.x], sh[2][threadIdx.x + s]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        R.block_part[3 * blockIdx.x + 0] = sh[0][0];
        R.block_part[3 * blockIdx.x + 1] = sh[1][0];
        R.block_part[3 * blockIdx.x + 2] = sh[2][0];
        __threadfence();
        unsigned ticket = atomicAdd(R.counter, 1u);
        last = ticket == gridDim.x - 1;
    }
    __syncthreads();
    if (!last || threadIdx.x >= 32) return;
    __threadfence();
    // last block, first warp: fixed-order sums over blocks and items
    const int lane = threadIdx.x;
    const volatile double* bp = R.block_part;
    double s_ab = 0.0, s_dt = 0.0, s_inf = 0.0, s_psi = 0.0;
    for (int b = lane; b < (int)gridDim.x; b += 32) {
        s_ab += bp[3 * b];
        s_dt += bp[3 * b + 1];
        s_inf = fmax(s_inf, bp[3 * b + 2]);
    }
    for (int it = lane; it < R.nitems; it += 32)
        if (R.item_active[it]) s_psi += R.psipart[it];
    for (int off = 16; off >= 1; off >>= 1) {
        s_ab += __shfl_xor_sync(FULLMASK, s_ab, off);
        s_dt += __shfl_xor_sync(FULLMASK, s_dt, off);
        s_inf = fmax(s_inf, __shfl_xor_sync(FULLMASK, s_inf, off));
        s_psi += __shfl_xor_sync(FULLMASK, s_psi, off);
    }
    if (lane == 0) {
        const double D = s_ab - s_psi;
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
                              int32_t m, int32_t n, float* Cs, int64_t ldcs)
{
    const int r = blockIdx.y;
    const float* src = C + (int64_t)perm[r] * ldc;
    float* dst = Cs + (int64_t)r * ldcs;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < ldcs; j += (int64_t)gridDim.x * blockDim.x)
        dst[j] = j < n ? src[j] : 0.f;
}

void launch_gather_rows(const float* C, int64_t ldc, const int32_t* perm, int32_t m, int32_t n, float* Cs,
                        int64_t ldcs, cudaStream_t st)
{
    int bx = (int)((ldcs + 255) / 256);
    if (bx > 64) bx = 64;
    for (int32_t r0 = 0; r0 < m; r0 += 65535) {
        int32_t rows = m - r0 < 65535 ? m - r0 : 65535;
        dim3 grid(bx, rows);
        k_gather_rows<<<grid, 256, 0, st>>>(C, ldc, perm + r0, rows, n, Cs + (int64_t)r0 * ldcs, ldcs);
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
