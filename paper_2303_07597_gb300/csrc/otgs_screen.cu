// otgs_screen.cu -- safe skipping of zero blocks (Sec. 3.2) and the set N of
// surely-nonzero blocks (Sec. 3.3), on the device.
//
// Arithmetic of the bounds (all FP32, fixed operation order, reproduced bit
// for bit by the oracle's replica of this rule):
//  * upper bound (Def. 1, Eq. 6), every operation rounded toward +inf so the
//    computed zbar is >= the exact bound (Lemma 1 survives rounding):
//      npos_l = sqrt(sum_i [alpha_i - alpha~_i]_+^2)         (rows of group l)
//      dbp_j  = [beta_j - beta~_j]_+
//      zbar   = (z~ + npos_l) + sqrt(g_l) * dbp_j
//    The block is skipped when zbar <= theta_skip_l = RD(theta - tau_l), with
//    tau_l = 2^-36 (sqrt(g_l) M + g_l theta) and M = max|alpha| + max|beta| +
//    max|alpha~| + max|beta~| + max c.  tau_l exceeds the rounding error of
//    the evaluation kernel's z (double-float f and S), so a skipped block also
//    evaluates to exactly zero there and screened == dense bit for bit.
//    The screen first applies the same formula to a whole 32-column tile with
//    the tile's largest z~ (formed once per snapshot) and largest dbp: every
//    step rounds up, so the tile's zbar bounds each column's, and a tile that
//    passes skips its columns outside N with no per-column read.  Only the
//    other tiles read z~ column by column; the skip decisions are the same.
//  * lower bound (Def. 2, Eq. 7), round-to-nearest (N only decides which
//    blocks are computed without a check, never a result):
//      zlow = k~ - ||dalpha_[l]|| - sqrt(g_l)|dbeta_j| - o~ - ||[dalpha_[l]]_-|| - sqrt(g_l)|[dbeta_j]_-|
//      k~ = sqrt(z~^2 + o~^2);  (l, j) in N  iff  zlow > theta.
// Group sums run lane-strided over the group's sorted rows (lane k takes rows
// k, k+32, ...) and then through a fixed xor tree (16, 8, 4, 2, 1).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "otgs_handle.cuh"

namespace otgs {

#define FULLMASK 0xffffffffu

struct ScreenArgs {
    int32_t m, n, L, ntiles, unit_words;
    const int32_t* goff;
    const double* alpha;     // sorted rows, current
    const double* alpha_s;   // sorted rows, snapshot
    const double* beta;
    const double* beta_s;
    const float* zt;         // L x ntiles*TW
    const float* zt_tile;    // L x ntiles: max of zt over each tile's columns (+inf with a NaN)
    const float* ot;
    const float* sg_ru;      // RU(sqrt(g_l))
    const float* sg_rn;      // RN(sqrt(g_l))
    float* gstat;            // [L][4]: npos (RU), nabs, nneg (RN)
    float* cstat;            // [3][ntiles*TW]: dbp (RU), |dbeta|, |[dbeta]_-| (RN), one array each;
                             // then [ntiles]: the largest dbp of each tile
    unsigned* gmax;          // [4] float bits, zeroed before the delta kernel
    float cmax;
    double theta;
    float theta_f;
    uint32_t* Nmask;         // [L][ntiles]
    uint32_t* skipmask;      // [L][ntiles]
    uint32_t* unit_need;     // [L][unit_words], zeroed before the screen kernel
    uint8_t* item_active;    // [nitems], zeroed before the screen kernel
    const int32_t* gpanel;
    const int32_t* pitem;
    const int32_t* pW;
    const int32_t* psplit;      // pieces of a panel's group (1: not split)
    unsigned long long* count;  // [0] in N, [1] checked, [2] skipped, [3] units needed, [4] C bytes read
    int32_t nitems;
    const int* gate;            // NULL, or a device flag: 0 = skip (batched solver trials)
    int32_t wl_build;           // 1: record each needed unit as a block set for the exact-sum kernels
    int32_t route;              // 0: chosen by size, 1: the bound pass, 2: the screen's block sets
    double wl_max;              // the screen's sets are taken when their rows x columns are at most this
};

__device__ __forceinline__ void atomic_max_pos(unsigned* addr, float v)
{
    atomicMax(addr, __float_as_uint(v));  // v >= 0: integer order == float order
}

// Per sorted row (the FP64 part of the group statistics, spread over the
// whole grid): (RU(RU(alpha - alpha~)) clamped at 0, RN(RN(alpha - alpha~)))
// as FP32, and the maxima of |alpha|, |alpha~| rounded up.
__global__ void k_delta_rows(const ScreenArgs S, float2* drow)
{
    if (S.gate && !*S.gate) return;
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (S.item_active && r < S.nitems) S.item_active[r] = 0;  // k_screen marks the items it needs
    float amax = 0.f, asmax = 0.f, bmax = 0.f, bsmax = 0.f;
    if (r < S.n) {  // the columns' maxima too, so that k_delta has M for theta_skip
        bmax = __double2float_ru(fabs(S.beta[r]));
        bsmax = __double2float_ru(fabs(S.beta_s[r]));
    }
    if (r < S.m) {
        const double al = S.alpha[r], as = S.alpha_s[r];
        const float du = __double2float_ru(__dsub_ru(al, as));
        drow[r] = make_float2(fmaxf(du, 0.f), __double2float_rn(__dsub_rn(al, as)));
        amax = __double2float_ru(fabs(al));
        asmax = __double2float_ru(fabs(as));
    }
    for (int off = 16; off >= 1; off >>= 1) {
        amax = fmaxf(amax, __shfl_xor_sync(FULLMASK, amax, off));
        asmax = fmaxf(asmax, __shfl_xor_sync(FULLMASK, asmax, off));
        bmax = fmaxf(bmax, __shfl_xor_sync(FULLMASK, bmax, off));
        bsmax = fmaxf(bsmax, __shfl_xor_sync(FULLMASK, bsmax, off));
    }
    if ((threadIdx.x & 31) == 0) {
        atomic_max_pos(S.gmax + 0, amax);
        atomic_max_pos(S.gmax + 1, bmax);
        atomic_max_pos(S.gmax + 2, asmax);
        atomic_max_pos(S.gmax + 3, bsmax);
    }
}

// theta_skip_l = RD(theta - 2^-36 (sqrt(g) M + g theta)), FP64 round-to-nearest inside.
__device__ __forceinline__ float theta_skip(const ScreenArgs& S, int g)
{
    const double M = __dadd_rn(__dadd_rn(__dadd_rn(__dadd_rn((double)__uint_as_float(S.gmax[0]),
                                                             (double)__uint_as_float(S.gmax[1])),
                                                    (double)__uint_as_float(S.gmax[2])),
                                           (double)__uint_as_float(S.gmax[3])),
                                  (double)S.cmax);
    const double tau = ldexp(__dadd_rn(__dmul_rn(__dsqrt_rn((double)g), M), __dmul_rn((double)g, S.theta)), -36);
    return __double2float_rd(__dsub_rn(S.theta, tau));
}

// Blocks [0, ceil(L/8)) take one group per warp (the sums, from the rows'
// FP32 values, and the group's theta_skip, once: FP64); the rest take columns.
__global__ void k_delta(const ScreenArgs S, int group_blocks, const float2* drow)
{
    if (S.gate && !*S.gate) return;
    if ((int)blockIdx.x < group_blocks) {
        const int l = blockIdx.x * 8 + (threadIdx.x >> 5);
        const int lane = threadIdx.x & 31;
        if (l >= S.L) return;
        const int r0 = S.goff[l], r1 = S.goff[l + 1];
        float pu = 0.f, a2 = 0.f, n2 = 0.f;
        // each lane visits rows r0 + lane, r0 + lane + 32, ... in that order
        // (the order the sums are defined in); loads sixteen rows ahead
        auto add = [&](float2 v) {
            const float dp = v.x, d = v.y;
            pu = __fadd_ru(pu, __fmul_ru(dp, dp));
            a2 = __fadd_rn(a2, __fmul_rn(d, d));
            const float dn = fminf(d, 0.f);
            n2 = __fadd_rn(n2, __fmul_rn(dn, dn));
        };
        int r = r0 + lane;
        for (; r + 32 * 15 < r1; r += 32 * 16) {
            float2 v[16];
#pragma unroll
            for (int q = 0; q < 16; q++) v[q] = drow[r + 32 * q];
#pragma unroll
            for (int q = 0; q < 16; q++) add(v[q]);
        }
        for (; r < r1; r += 32) add(drow[r]);
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) {
            pu = __fadd_ru(pu, __shfl_xor_sync(FULLMASK, pu, off));
            a2 = __fadd_rn(a2, __shfl_xor_sync(FULLMASK, a2, off));
            n2 = __fadd_rn(n2, __shfl_xor_sync(FULLMASK, n2, off));
        }
        if (lane == 0) {
            S.gstat[4 * l + 0] = __fsqrt_ru(pu);
            S.gstat[4 * l + 1] = __fsqrt_rn(a2);
            S.gstat[4 * l + 2] = __fsqrt_rn(n2);
            S.gstat[4 * l + 3] = theta_skip(S, r1 - r0);  // (the maxima are complete: k_delta_rows)
        }
        return;
    }
    const int j = (blockIdx.x - group_blocks) * blockDim.x + threadIdx.x;
    if (j >= S.ntiles * TW) return;
    float dbp = 0.f, dba = 0.f, dbn = 0.f;
    if (j < S.n) {
        const double be = S.beta[j], bs = S.beta_s[j];
        dbp = fmaxf(__double2float_ru(__dsub_ru(be, bs)), 0.f);
        const float d = __double2float_rn(__dsub_rn(be, bs));
        dba = fabsf(d);
        dbn = fabsf(fminf(d, 0.f));
    }
    const int ldz = S.ntiles * TW;
    S.cstat[j] = dbp;
    S.cstat[ldz + j] = dba;
    S.cstat[2 * ldz + j] = dbn;
    // a warp holds one tile's columns (whole warps return above): the tile's largest dbp
    float tm = dbp;
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) tm = fmaxf(tm, __shfl_xor_sync(FULLMASK, tm, off));
    if ((threadIdx.x & 31) == 0) S.cstat[3 * ldz + (j >> 5)] = tm;
}

// After a snapshot: per unit (group l, tile jt) the largest z~ over the
// tile's columns (columns past n count as 0; a NaN makes it +inf), for the
// screen's tile-level test.  One warp per unit.
__global__ void k_zt_tiles(const float* zt, float* zt_tile, int64_t units, int ntiles, int n, const int* gate)
{
    if (gate && !*gate) return;
    const int64_t u = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (u >= units) return;
    const int lane = threadIdx.x & 31;
    const int j = (int)(u % ntiles) * TW + lane;
    float z = j < n ? zt[u * TW + lane] : 0.f;
    if (z != z) z = INFINITY;
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) z = fmaxf(z, __shfl_xor_sync(FULLMASK, z, off));
    if (lane == 0) zt_tile[u] = z;
}


// Alg. 2's skip test (Eq. 6, Lemma 2) for every block outside N.  A warp
// takes the 32 units (l, 32-column tile) of one unit_need word, lane t tile
// t; a tile that fails the tile-level test is screened column by column
// (lane = column), and lane t keeps tile t's skip word, writes it and marks
// its items.  With wl_build, every unit with a block left is also recorded
// as a block set for the exact-sum kernels (its group's rows x the tile's
// columns not skipped): the warps of a CTA count their sets and column tasks,
// one atomic per counter and CTA hands out their places, and each lane
// writes its tile's set; the rows x columns of the sets are summed, and the
// last CTA to finish picks the route.  Statistics are summed per CTA before
// one atomic add each.
constexpr int SCREEN_WARPS = 8;
constexpr int SCREEN_TB = 8;  // tiles whose loads a warp issues together

__device__ void pick_route(const ScreenArgs& S, EvalCtl* ctl, unsigned long long* fcount);

__global__ void __launch_bounds__(SCREEN_WARPS * 32) k_screen(const ScreenArgs S, const EvalArgs E)
{
    if (S.gate && !*S.gate) return;
    __shared__ unsigned long long csum[SCREEN_WARPS][4];
    __shared__ int wcnt[3][SCREEN_WARPS];  // a round's short sets, tall sets, tall column tasks per warp
    __shared__ int wbase[3][SCREEN_WARPS]; // the index of each warp's first one
    __shared__ bool last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    const int64_t ntask = (int64_t)S.L * S.unit_words;
    unsigned long long c0 = 0, c1 = 0, c2 = 0, c3 = 0, work = 0, wcols = 0;
    // rounds of SCREEN_WARPS tasks, the same count in every warp of the CTA
    for (int64_t base = (int64_t)blockIdx.x * SCREEN_WARPS; base < ntask;
         base += (int64_t)gridDim.x * SCREEN_WARPS) {
        const int64_t task = base + warp;
        const bool have = task < ntask;  // (uniform in the warp)
        const int l = have ? (int)(task / S.unit_words) : 0, w = have ? (int)(task % S.unit_words) : 0;
        const int gs = S.goff[l], ge = S.goff[l + 1];
        const int g = have ? ge - gs : 0;
        const float th = S.gstat[4 * l + 3], npos = S.gstat[4 * l], sg = S.sg_ru[l];
        const int jt1 = min(32 * w + 32, S.ntiles);
        const int ldz = S.ntiles * TW;
        // lane t: tile jt = 32 w + t; its word of N, its existing columns (none
        // in an empty group) and the tile-level test: with z~max and dbpmax the
        // tile's largest z~ and dbp, RU((z~max + npos) + sg dbpmax) <= theta_skip
        // implies the block test below for each of its columns (every operation
        // rounds up, so the bound grows with each operand), so the tile's skip
        // word is then its columns outside N without reading their z~
        const int jt = 32 * w + lane;
        const bool tv = have && jt < jt1;
        const int64_t tq = (int64_t)l * S.ntiles + jt;
        const uint32_t my_N = tv ? __ldg(S.Nmask + tq) : 0u;
        const int cols = min(TW, S.n - jt * TW);
        const uint32_t my_valid = (tv && g > 0) ? (cols >= TW ? FULLMASK : (1u << cols) - 1u) : 0u;
        bool pass = false;
        if (my_valid) {
            const float zb = __fadd_ru(__fadd_ru(__ldg(S.zt_tile + tq), npos), __fmul_ru(sg, __ldg(S.cstat + 3 * ldz + jt)));
            pass = zb <= th;
        }
        uint32_t my_skip = pass ? my_valid & ~my_N : 0u;
        // the other tiles column by column (Eq. 6), lane = column, SCREEN_TB
        // tiles' loads issued together
        uint32_t todo = __ballot_sync(FULLMASK, my_valid != 0u && !pass);
        while (todo) {
            int tl[SCREEN_TB];
            float zv[SCREEN_TB], dv[SCREEN_TB];
#pragma unroll
            for (int q = 0; q < SCREEN_TB; q++) {
                tl[q] = todo ? __ffs(todo) - 1 : -1;
                todo &= todo - 1u;
                const int j = (32 * w + tl[q]) * TW + lane;
                const bool ok = tl[q] >= 0 && j < S.n;
                zv[q] = ok ? __ldg(S.zt + (int64_t)l * ldz + j) : 0.f;
                dv[q] = ok ? __ldg(S.cstat + j) : 0.f;
            }
#pragma unroll
            for (int q = 0; q < SCREEN_TB; q++) {
                if (tl[q] < 0) break;  // (uniform)
                const uint32_t Nv = __shfl_sync(FULLMASK, my_N, tl[q]);
                const int j = (32 * w + tl[q]) * TW + lane;
                bool skip = false;
                if (j < S.n && !((Nv >> lane) & 1u)) {
                    const float zbar = __fadd_ru(__fadd_ru(zv[q], npos), __fmul_ru(sg, dv[q]));
                    skip = zbar <= th;
                }
                const uint32_t skipw = __ballot_sync(FULLMASK, skip);
                if (lane == tl[q]) my_skip = skipw;
            }
        }
        const uint32_t my_need = my_valid & ~my_skip;
        // every lane its own tile: the skip word, the items that hold it, the statistics
        if (tv) {
            S.skipmask[(int64_t)l * S.ntiles + jt] = my_skip;
            if (my_need) {
                // the item of (l, tile) in every piece of the group (same value from every writer)
                const int p = S.gpanel[l];
                for (int k = 0; k < S.psplit[p]; k++) S.item_active[S.pitem[p + k] + (jt * TW) / S.pW[p]] = 1;
            }
            c0 += __popc(my_N & my_valid);
            c1 += __popc(~my_N & my_valid);
            c2 += __popc(my_skip);
            c3 += my_need ? 1ull : 0ull;
        }
        const uint32_t needword = __ballot_sync(FULLMASK, my_need != 0u);
        if (lane == 0 && have) S.unit_need[(int64_t)l * S.unit_words + w] = needword;
        if (!S.wl_build) continue;  // (uniform in the kernel)
        // the units with a block left as block sets
        const bool tall = g > XTALL_ROWS;
        const int nc = __popc(my_need);
        int cs = nc;  // inclusive scan of the columns over the lanes
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int v = __shfl_up_sync(FULLMASK, cs, off);
            if (lane >= off) cs += v;
        }
        const int ctot = __shfl_sync(FULLMASK, cs, 31);
        if (lane == 0) {
            wcnt[0][warp] = tall ? 0 : __popc(needword);
            wcnt[1][warp] = tall ? __popc(needword) : 0;
            wcnt[2][warp] = tall && E.use_ct ? ctot : 0;
        }
        work += (unsigned long long)g * (unsigned long long)ctot;
        wcols += (unsigned long long)ctot;
        __syncthreads();
        if (threadIdx.x < 3) {
            const int k = threadIdx.x;
            int tot = 0;
            for (int q = 0; q < SCREEN_WARPS; q++) {
                wbase[k][q] = tot;
                tot += wcnt[k][q];
            }
            if (tot) {
                const int b0 = atomicAdd(k == 0 ? &E.ctl->nxent : (k == 1 ? &E.ctl->nxtall : &E.ctl->ntcol), tot);
                for (int q = 0; q < SCREEN_WARPS; q++) wbase[k][q] += b0;
            }
        }
        __syncthreads();
        if (my_need) {
            const int e = wbase[tall ? 1 : 0][warp] + __popc(needword & lt);
            const int tb = wbase[2][warp] + (cs - nc);
            if (e >= (tall ? E.xtall_cap : E.xent_cap) || (tall && E.use_ct && tb + nc > E.xtcol_cap)) {
                atomicOr(E.err, 4);  // the capacities hold every (group, column) once: not reached
                continue;
            }
            XEntry& x = (tall ? E.xtall : E.xent)[e];
            x.gstart = gs;
            x.gend = ge;
            x.colg0 = jt * TW;
            x.prob = 0;
            x.l = l;
            x.mask = my_need;
            x.tbase = tb;
            if (tall && E.use_ct)
                for (int i = 0; i < nc; i++) E.xtmap[tb + i] = (uint32_t)e;
        }
    }
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        c0 += __shfl_xor_sync(FULLMASK, c0, off);
        c1 += __shfl_xor_sync(FULLMASK, c1, off);
        c2 += __shfl_xor_sync(FULLMASK, c2, off);
        c3 += __shfl_xor_sync(FULLMASK, c3, off);
    }
    if (lane == 0) {
        csum[warp][0] = c0;
        csum[warp][1] = c1;
        csum[warp][2] = c2;
        csum[warp][3] = c3;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        unsigned long long v = 0;
        for (int q = 0; q < SCREEN_WARPS; q++) v += csum[q][threadIdx.x];
        if (v) atomicAdd(S.count + threadIdx.x, v);
    }
    if (!S.wl_build) return;
    if (lane == 0 && work) {
        atomicAdd(&E.ctl->wl_work, work);
        atomicAdd(&E.ctl->wl_cols, wcols);
    }
    // the last CTA to finish picks the route (every CTA's sums are in)
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(&E.ctl->wl_done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        pick_route(S, E.ctl, E.fcount);
    }
}

// The route of a screened evaluation (the last CTA of k_screen, which
// recorded every needed unit
// as a block set for the exact-sum kernels): when their rows x columns are few
// (at most wl_max: then reading just those blocks from the transposed copy
// costs less than a bound pass over every needed tile) the evaluation takes
// them as they are and the bound pass and its kernels stand down (ctl->wl).
// Otherwise the sets are dropped and the bound pass flags its own.  Either
// way every block with s > 0 is formed by the same exact-sum kernels, so the
// route changes no result.
__device__ void pick_route(const ScreenArgs& S, EvalCtl* ctl, unsigned long long* fcount)
{
    const double w = (double)ctl->wl_work;
    const bool wl = S.wl_build && (S.route == 2 || (S.route == 0 && w <= S.wl_max));
    ctl->wl = wl ? 1 : 0;
    if (wl) {
        S.count[4] += (unsigned long long)(4.0 * w);  // the blocks' bytes of C
        if (fcount) *fcount += ctl->wl_cols;
    } else {
        ctl->nxent = 0;
        ctl->nxtall = 0;
        ctl->ntcol = 0;
    }
}

// Alg. 1, every r iterations: N from the lower bound against the current snapshot.
__global__ void k_build_N(const ScreenArgs S)
{
    const int64_t u = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (u >= (int64_t)S.L * S.ntiles) return;
    const int l = (int)(u / S.ntiles), jt = (int)(u % S.ntiles);
    const int g = S.goff[l + 1] - S.goff[l];
    const int j = jt * TW + lane;
    bool inN = false;
    if (j < S.n && g > 0) {
        const int64_t q = (int64_t)l * S.ntiles * TW + j;
        const float z = S.zt[q], o = S.ot[q];
        const float kt = __fsqrt_rn(__fadd_rn(__fmul_rn(z, z), __fmul_rn(o, o)));
        const float sg = S.sg_rn[l];
        float zl = __fsub_rn(kt, S.gstat[4 * l + 1]);
        zl = __fsub_rn(zl, __fmul_rn(sg, S.cstat[S.ntiles * TW + j]));
        zl = __fsub_rn(zl, o);
        zl = __fsub_rn(zl, S.gstat[4 * l + 2]);
        zl = __fsub_rn(zl, __fmul_rn(sg, S.cstat[2 * S.ntiles * TW + j]));
        inN = zl > S.theta_f;
    }
    const uint32_t w = __ballot_sync(FULLMASK, inN);
    if (lane == 0) S.Nmask[u] = w;
}

// ------------------------------------------------------------------- host
ScreenArgs make_screen_args(Handle* h)
{
    ScreenArgs s;
    memset(&s, 0, sizeof(s));
    s.m = (int32_t)h->m; s.n = (int32_t)h->n; s.L = h->L; s.ntiles = h->ntiles; s.unit_words = h->unit_words;
    s.goff = h->dp.goff;
    s.alpha = h->alpha_eval; s.alpha_s = h->alpha_snap;
    s.beta = nullptr; s.beta_s = h->beta_snap;
    s.zt = h->zt; s.ot = h->ot; s.zt_tile = h->zt_tile;
    s.sg_ru = h->sg_ru; s.sg_rn = h->sg_rn;
    s.gstat = h->gstat; s.cstat = h->cstat; s.gmax = h->gmax;
    s.cmax = h->cmax;
    s.theta = h->prm.mu * h->prm.gamma;
    s.theta_f = (float)s.theta;
    s.Nmask = h->Nmask; s.skipmask = h->skipmask; s.unit_need = h->unit_need; s.item_active = h->item_active;
    s.gpanel = h->dp.gpanel; s.pitem = h->dp.pitem; s.pW = h->dp.pW; s.psplit = h->dp.psplit;
    s.count = h->dcount;
    s.nitems = h->hp.nitems();
    s.gate = h->eval_gate;
    return s;
}

bool Handle::ensure_screen()
{
    if (screen_alloc) return true;
    const size_t ldz = (size_t)ntiles * TW;
    zt = (float*)dalloc(sizeof(float) * (size_t)L * ldz, "zt");
    zt_tile = (float*)dalloc(sizeof(float) * (size_t)L * ntiles, "zt_tile");
    ot = (float*)dalloc(sizeof(float) * (size_t)L * ldz, "ot");
    alpha_snap = (double*)dalloc(sizeof(double) * m, "alpha_snap");
    beta_snap = (double*)dalloc(sizeof(double) * n, "beta_snap");
    Nmask = (uint32_t*)dalloc(sizeof(uint32_t) * (size_t)L * ntiles, "Nmask");
    skipmask = (uint32_t*)dalloc(sizeof(uint32_t) * (size_t)L * ntiles, "skipmask");
    unit_need = (uint32_t*)dalloc(sizeof(uint32_t) * (size_t)L * unit_words, "unit_need");
    item_active = (uint8_t*)plan_alloc((size_t)hp.nitems(), "item_active");
    stage_m8 = (uint8_t*)plan_alloc((size_t)hp.nstages * STAGE_ROWS, "stage masks");
    stage_need = (uint32_t*)plan_alloc(sizeof(uint32_t) * (size_t)((hp.nstages + 31) / 32), "stages needed");
    if (!stage_m8 || !stage_need) return false;
    gstat = (float*)dalloc(sizeof(float) * 4 * (size_t)L, "gstat");
    drow = (float2*)dalloc(sizeof(float2) * (size_t)m, "per-row changes of alpha");
    if (!drow) return false;
    cstat = (float*)dalloc(sizeof(float) * 4 * ldz, "cstat");
    gmax = (unsigned*)dalloc(sizeof(unsigned) * 8, "gmax");
    dcount = (unsigned long long*)dalloc(sizeof(unsigned long long) * 8, "dcount");
    if (!zt || !zt_tile || !ot || !alpha_snap || !beta_snap || !Nmask || !skipmask || !unit_need || !item_active || !gstat ||
        !cstat || !gmax || !dcount)
        return false;
    std::vector<float> ru(L), rn(L);
    for (int32_t l = 0; l < L; l++) {
        const double g = (double)(hp.goff[l + 1] - hp.goff[l]);
        const double s = std::sqrt(g);
        float f = (float)s;
        rn[l] = f;
        if ((double)f < s) f = std::nextafter(f, INFINITY);
        ru[l] = f;
    }
    sg_ru = (float*)dalloc(sizeof(float) * L, "sg_ru");
    sg_rn = (float*)dalloc(sizeof(float) * L, "sg_rn");
    if (!sg_ru || !sg_rn) return false;
    if (!ck(cudaMemcpyAsync(sg_ru, ru.data(), sizeof(float) * L, cudaMemcpyHostToDevice, st), "sg upload"))
        return false;
    if (!ck(cudaMemcpyAsync(sg_rn, rn.data(), sizeof(float) * L, cudaMemcpyHostToDevice, st), "sg upload"))
        return false;
    if (!ck(cudaMemsetAsync(dcount, 0, sizeof(unsigned long long) * 8, st), "memset")) return false;
    if (!ck(cudaMemsetAsync(Nmask, 0, sizeof(uint32_t) * (size_t)L * ntiles, st), "memset")) return false;
    if (!ck(cudaStreamSynchronize(st), "screen alloc sync")) return false;
    screen_alloc = true;
    return true;
}

// The tile maxima of z~ (k_screen's tile-level test) from the current z~.
bool Handle::zt_tiles()
{
    const int64_t units = (int64_t)L * ntiles;
    k_zt_tiles<<<(unsigned)((units + 7) / 8), 256, 0, st>>>(zt, zt_tile, units, ntiles, (int)n, eval_gate);
    return ck(cudaGetLastError(), "zt tiles launch");
}

// As Alg. 1 starts: the first snapshot is taken at alpha~ = beta~ = 0 with N empty.
bool Handle::zero_snapshot()
{
    cudaMemsetAsync(alpha_snap, 0, sizeof(double) * m, st);
    cudaMemsetAsync(beta_snap, 0, sizeof(double) * n, st);
    cudaMemsetAsync(Nmask, 0, sizeof(uint32_t) * (size_t)L * ntiles, st);
    if (!eval_dense(alpha_snap, true, beta_snap, nullptr, nullptr, nullptr, true)) return false;
    snap_valid = true;
    stats_host.snapshots++;
    return true;
}

// Delta statistics of (alpha_eval, beta) against the snapshot.
static void launch_delta(Handle* h, const double* beta)
{
    ScreenArgs s = make_screen_args(h);
    s.beta = beta;
    if (!h->eval_gate) cudaMemsetAsync(h->gmax, 0, sizeof(unsigned) * 4, h->st);  // else cleared by the trial gate
    const int gblocks = (h->L + 7) / 8;
    const int cblocks = (h->ntiles * TW + 255) / 256;
    const int64_t nt = std::max<int64_t>(std::max<int64_t>(h->m, h->n), h->hp.nitems());
    k_delta_rows<<<(unsigned)((nt + 255) / 256), 256, 0, h->st>>>(s, h->drow);
    k_delta<<<gblocks + cblocks, 256, 0, h->st>>>(s, gblocks, h->drow);
}

bool Handle::snapshot_at(const double* alpha, bool alpha_sorted, const double* beta, bool build_N,
                         double* out_caller, double* G_sorted, const double* dir)
{
    if (!ensure_screen()) return false;
    if (!snap_valid && !zero_snapshot()) return false;
    prep(alpha, alpha_sorted, beta);
    if (build_N && prm.use_lower_bound) {
        launch_delta(this, beta);
        ScreenArgs s = make_screen_args(this);
        s.beta = beta;
        const int64_t units = (int64_t)L * ntiles;
        k_build_N<<<(unsigned)((units + 7) / 8), 256, 0, st>>>(s);
    } else if (build_N) {
        cudaMemsetAsync(Nmask, 0, sizeof(uint32_t) * (size_t)L * ntiles, st);
    }
    if (!eval_dense(alpha_eval, true, beta, out_caller, G_sorted, dir, true)) return false;
    cudaMemcpyAsync(alpha_snap, alpha_eval, sizeof(double) * m, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(beta_snap, beta, sizeof(double) * n, cudaMemcpyDeviceToDevice, st);
    stats_host.snapshots++;
    return ck(cudaGetLastError(), "snapshot launch");
}

bool Handle::eval_screened(const double* alpha, bool alpha_sorted, const double* beta, double* out_caller,
                           double* G_sorted, const double* dir)
{
    if (!ensure_screen()) return false;
    if (!snap_valid && !zero_snapshot()) return false;
    prep(alpha, alpha_sorted, beta);
    if (!eval_gate) stats_host.kernels += 1;
    return eval_screened_prepped(beta, G_sorted, dir, out_caller);
}

bool Handle::eval_screened_prepped(const double* beta, double* G_sorted, const double* dir, double* out_caller)
{
    if (!ensure_screen()) return false;
    if (!snap_valid) return fail(OTGS_EINVAL, "screened evaluation without a snapshot");
    launch_delta(this, beta);
    ScreenArgs s = make_screen_args(this);
    s.beta = beta;
    EvalArgs e = eval_args(item_active, unit_need, false);
    e.stage_m8 = stage_m8;
    e.stage_need = stage_need;
    e.c_streamed = dcount + 4;
    s.wl_build = e.use_ct && dbg_route != 1;
    s.route = (int32_t)dbg_route;
    s.wl_max = WL_FRACTION * (double)m * (double)n;
    const int64_t tasks = (int64_t)L * unit_words;
    const int sblocks = (int)std::min<int64_t>((tasks + SCREEN_WARPS - 1) / SCREEN_WARPS, 16LL * n_sm);
    // (without the block sets the control word's zero route is the bound pass)
    k_screen<<<sblocks, SCREEN_WARPS * 32, 0, st>>>(s, e);
    launch_stage_masks(e, n_sm, st);
    const int nk = eval_launch(e, std::min(CTAS_PER_SM * n_sm, hp.nitems()));
    ReduceArgs r = reduce_args(item_active, out_caller, G_sorted, dir, beta);
    launch_reduce(r, st);
    if (!eval_gate) {
        count_screened_evals(1);
        // and deltas (2), screen, stage masks, reduction
        stats_host.kernels += nk + 5;
    }
    return ck(cudaGetLastError(), "screened eval launch");
}

bool Handle::collect_stats()
{
    if (!screen_alloc) return true;
    unsigned long long c[8];
    if (!ck(cudaMemcpy(c, dcount, sizeof(c), cudaMemcpyDeviceToHost), "stats D2H")) return false;
    stats_host.blocks_in_N = (int64_t)c[0];
    stats_host.blocks_checked = (int64_t)c[1];
    stats_host.blocks_skipped = (int64_t)c[2];
    stats_host.units_computed = dense_units + (int64_t)c[3];
    stats_host.c_bytes = dense_cbytes + (double)c[4];
    return true;
}

void Handle::reset_device_stats()
{
    dense_units = 0;
    dense_cbytes = 0.0;
    if (screen_alloc) cudaMemsetAsync(dcount, 0, sizeof(unsigned long long) * 8, st);
}

}  // namespace otgs

using namespace otgs;

extern "C" {

int ot_gs_grad_screened(ot_gs* hh, const double* alpha, const double* beta, double* out, uint32_t* skip_mask)
{
    if (!hh) return OTGS_EINVAL;
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!single_problem(h)) return OTGS_EINVAL;
    if (!alpha || !beta || !out) { h->fail(OTGS_EINVAL, "NULL pointer"); return OTGS_EINVAL; }
    if (!h->eval_screened(alpha, false, beta, out, nullptr, nullptr)) return h->last_code;
    if (skip_mask &&
        !h->ck(cudaMemcpyAsync(skip_mask, h->skipmask, sizeof(uint32_t) * (size_t)h->L * h->ntiles,
                               cudaMemcpyDeviceToDevice, h->st), "skip mask copy"))
        return OTGS_ECUDA;
    return OTGS_OK;
}

int ot_gs_snapshot(ot_gs* hh, const double* alpha, const double* beta, int build_N, double* out)
{
    if (!hh) return OTGS_EINVAL;
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!single_problem(h)) return OTGS_EINVAL;
    if (!alpha || !beta) { h->fail(OTGS_EINVAL, "NULL pointer"); return OTGS_EINVAL; }
    if (!h->snapshot_at(alpha, false, beta, build_N != 0, out, nullptr, nullptr)) return h->last_code;
    return OTGS_OK;
}

int ot_gs_get_screen_state(ot_gs* hh, float* zt, float* ot, double* alpha_s, double* beta_s, uint32_t* N_mask)
{
    if (!hh) return OTGS_EINVAL;
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!single_problem(h)) return OTGS_EINVAL;
    if (!h->ensure_screen()) return h->last_code;
    if (!h->snap_valid) { h->fail(OTGS_EINVAL, "no snapshot yet"); return OTGS_EINVAL; }
    const size_t lz = (size_t)h->L * h->ntiles * TW;
    if (zt && !h->ck(cudaMemcpyAsync(zt, h->zt, sizeof(float) * lz, cudaMemcpyDeviceToDevice, h->st), "copy"))
        return OTGS_ECUDA;
    if (ot && !h->ck(cudaMemcpyAsync(ot, h->ot, sizeof(float) * lz, cudaMemcpyDeviceToDevice, h->st), "copy"))
        return OTGS_ECUDA;
    if (alpha_s) launch_permute_f64(h->alpha_snap, h->dp.perm, (int32_t)h->m, alpha_s, false, h->st);
    if (beta_s && !h->ck(cudaMemcpyAsync(beta_s, h->beta_snap, sizeof(double) * h->n, cudaMemcpyDeviceToDevice,
                                         h->st), "copy"))
        return OTGS_ECUDA;
    if (N_mask && !h->ck(cudaMemcpyAsync(N_mask, h->Nmask, sizeof(uint32_t) * (size_t)h->L * h->ntiles,
                                         cudaMemcpyDeviceToDevice, h->st), "copy"))
        return OTGS_ECUDA;
    return h->ck(cudaGetLastError(), "get_screen_state") ? OTGS_OK : OTGS_ECUDA;
}

}  // extern "C"
