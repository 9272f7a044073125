// otgs_stream.cu -- the evaluation kernel: one pass over C per evaluation of
// the dual (Eq. 4) and its gradient (Eq. 5), fed by TMA.
//
// Persistent, one CTA per SM, warp-specialised:
//  * a producer warp takes work items (host-built descriptors, fetched one
//    item ahead) from a global counter and streams each stage -- up to
//    STAGE_ROWS rows x STAGE_COLS columns of C as 2D TMA boxes, plus the
//    rows' alpha pairs and the columns' beta pairs as bulk copies -- into a
//    ring of NSTAGES shared-memory stages completed by mbarrier transaction
//    counts;
//  * eight consumer warps evaluate the stage out of shared memory, lane k
//    owning columns k and k + 32 of the stage, and release it.
// A stage holds a small panel (whole groups of <= STAGE_ROWS rows; each warp
// walks a contiguous run of whole groups) or STAGE_ROWS rows of one big group
// (each warp takes 16 rows; per-column partial sums meet in shared memory in
// warp order).  A big group's tile pair spans ceil(g / STAGE_ROWS) stages; they
// stay in the ring for the second pass when they fit, else the second pass
// re-reads the rows from L2.
//
// Per block (group l, column j): pass A forms f = alpha_i + beta_j - c_ij only
// where the cheap bound c_ij < A'_i + B'_j says f may be positive (A', B' are
// alpha, beta rounded up by a relative 2^-22, so no positive f is missed), in
// double-float with TwoSum, and sums S = ||[f_[l]]_+||^2 and P = sum [f_[l]]_+;
// then the shrink s = [z - theta]_+ / (gamma z) and psi = [z - theta]_+^2 /
// (2 gamma) of Eq. 5; pass B adds s [f]_+ into the row sums (one warp sum per
// row).  Row, column and psi partial sums go to per-item buffers that the
// reduction kernel adds in a fixed order.
//
// Every wait is on an mbarrier and gives up after WAIT_NS (the consumer warps'
// own barrier is an mbarrier too); on timeout the kernel records an error in
// A.err, the producer waits (bounded) for the copies it issued, and all warps
// return.
#include <mutex>
#include <string>

#include "otgs_internal.cuh"

namespace otgs {

#define FULLMASK 0xffffffffu

namespace {

constexpr int CONSUMERS = 8;
constexpr int THREADS = (CONSUMERS + 1) * 32;
constexpr int SC = STAGE_COLS;                         // columns per stage
constexpr int WROWS = STAGE_ROWS / CONSUMERS;          // big stages: rows per consumer warp
constexpr uint32_t ROW_BYTES = SC * 4;                 // a TMA box row, zero-filled past column n
constexpr unsigned long long WAIT_NS = 2000000000ull;  // give up a wait after 2 s

enum : int { H_FIRST = 1, H_LAST = 2, H_TERM = 4, H_BIG_HELD = 8, H_SKIP = 16 };

// Everything the consumers need about a stage, written by the producer: the
// item's descriptor plus the stage's own fields.
struct StageHdr {
    ItemDesc d;
    int tile, sidx, nst, flags;
    int a_shift;  // offset of the stage's row 0 in arow[]
    int pad[3];
};

struct Smem {
    float stage[NSTAGES][STAGE_ROWS * SC];   // NSTAGES x 32 KB; stage row r at [r * SC]
    float2 arow[NSTAGES][STAGE_ROWS + 2];    // (alpha hi, lo) of the stage's rows; row r at [r + a_shift]
    float2 colB[NSTAGES][SC];                // (beta hi, lo) of the stage's columns
    float colP[NSTAGES][SC];                 // B' of the stage's columns
    int4 gstage[NSTAGES][PANEL_MAX_GROUPS];  // first stage of a small item: the panel's group entries
    int4 ginfo[PANEL_MAX_GROUPS];            // small item: {group, first sorted row, rows, row in panel}
    uint64_t full[NSTAGES];
    uint64_t empty[NSTAGES];
    uint64_t cbar;  // barrier of the consumer warps
    StageHdr hdr[NSTAGES];
    float colacc[CONSUMERS][SMALL_CHUNK];  // small item: per-warp column sums
    float rowacc[BIG_SMEM_ROWS];           // row sums of the current item
    float4 red[CONSUMERS][SC];             // big tiles: per-warp (S_h, S_l, P_h, P_l) per column
    float redO[CONSUMERS][SC];
    double psi_w[CONSUMERS];
    int anyw[CONSUMERS];
};

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect(uint64_t* b, uint32_t bytes)
{
    asm volatile("mbarrier.expect_tx.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* b)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(su32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long gtime()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Wait for the phase with the given parity to complete; false after WAIT_NS.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity)
{
    if (mbar_try(b, parity)) return true;
    const unsigned long long t0 = gtime();
    for (;;) {
        for (int i = 0; i < 64; i++)
            if (mbar_try(b, parity)) return true;
        if (gtime() - t0 > WAIT_NS) return false;
    }
}

// 1D bulk copy (both addresses 16-byte aligned, bytes a multiple of 16).
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(su32(dst)),
        "l"(src), "r"(bytes), "r"(su32(bar))
        : "memory");
}

// One TMA box: rows [y, y + 2^k) x columns [x, x + SC) of C into dst.
__device__ __forceinline__ void tma_box(const TmaMaps& T, int k, float* dst, int x, int y, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(su32(dst)),
        "l"(reinterpret_cast<uint64_t>(&T.box[k])), "r"(x), "r"(y), "r"(su32(bar))
        : "memory");
}

// Rows [y, y + rows) (rows <= 2^(TMA_BOXES-1)) into dst rows [0, rows): one
// box per set bit of rows, so exactly the requested rows are read.
__device__ __forceinline__ void tma_rows(const TmaMaps& T, float* dst, int x, int y, int rows, uint64_t* bar)
{
    int off = 0;
#pragma unroll
    for (int k = TMA_BOXES - 1; k >= 0; k--)
        if (rows & (1 << k)) {
            tma_box(T, k, dst + off * SC, x, y + off, bar);
            off += 1 << k;
        }
}

// ---------------------------------------------------------------- arithmetic
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

// f = (ah + al) + (bh + bl) - c as a float pair, |error| ~ 2^-46 (|alpha| + |beta| + c).
__device__ __forceinline__ void f_exact(float ah, float al, float bh, float bl, float c, float& fh, float& fl)
{
    float s1, e1, s2, e2;
    two_sum(ah, -c, s1, e1);
    two_sum(s1, bh, s2, e2);
    float t = __fadd_rn(__fadd_rn(e1, e2), __fadd_rn(al, bl));
    fh = __fadd_rn(s2, t);
    fl = __fsub_rn(t, __fsub_rn(fh, s2));
}

struct Acc {
    float Sh, Sl, Ph, Pl;  // S = sum p^2 and P = sum p, double-float
};

// S += p^2 and P += p for p = (fh, fl) > 0.
__device__ __forceinline__ void acc_p(float fh, float fl, Acc& a)
{
    float q = __fmul_rn(fh, fh);
    float ql = fmaf(fh, fh, -q);
    ql = fmaf(2.f * fh, fl, ql);
    df_add(a.Sh, a.Sl, q, ql);
    df_add(a.Ph, a.Pl, fh, fl);
}

// Eq. 5 for one block from S = ||[f_[l]]_+||^2: the shrink factor
// s = [z - theta]_+ / (gamma z); psi = [z - theta]_+^2 / (2 gamma).
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
__device__ __forceinline__ float z_up(float Sh, float Sl) { return __fsqrt_ru(fmaxf(__fadd_ru(Sh, Sl), 0.f)); }

// This lane's two columns of the stage: k and k + 32.
struct Col2 {
    float bh0, bl0, bp0, bh1, bl1, bp1;
};

__device__ __forceinline__ Col2 load_cols(const Smem& S, int slot, int lane)
{
    Col2 c;
    const float2 u = S.colB[slot][lane], v = S.colB[slot][lane + 32];
    c.bh0 = u.x; c.bl0 = u.y; c.bh1 = v.x; c.bl1 = v.y;
    c.bp0 = S.colP[slot][lane];
    c.bp1 = S.colP[slot][lane + 32];
    return c;
}

// Pass A for one row: c0, c1 in this lane's columns.
template <bool SNAP>
__device__ __forceinline__ bool row_a(float2 a2, float c0, float c1, const Col2& cl, Acc& a0, Acc& a1, float& O0,
                                      float& O1)
{
    if (SNAP) {
        const float x0 = fminf(__fsub_rn(__fadd_rn(a2.x, cl.bh0), c0), 0.f);
        const float x1 = fminf(__fsub_rn(__fadd_rn(a2.x, cl.bh1), c1), 0.f);
        O0 = fmaf(x0, x0, O0);
        O1 = fmaf(x1, x1, O1);
    }
    const float ap = bound_up(a2.x);
    bool any = false;
    if (c0 < __fadd_rn(ap, cl.bp0)) {
        float fh, fl;
        f_exact(a2.x, a2.y, cl.bh0, cl.bl0, c0, fh, fl);
        if (fh > 0.f) { acc_p(fh, fl, a0); any = true; }
    }
    if (c1 < __fadd_rn(ap, cl.bp1)) {
        float fh, fl;
        f_exact(a2.x, a2.y, cl.bh1, cl.bl1, c1, fh, fl);
        if (fh > 0.f) { acc_p(fh, fl, a1); any = true; }
    }
    return any;
}

// Pass B for one row: s0 [f]_+ + s1 [f]_+ over this lane's columns.
__device__ __forceinline__ float row_b(float2 a2, float c0, float c1, const Col2& cl, float s0, float s1)
{
    const float ap = bound_up(a2.x);
    float rs = 0.f;
    if (s0 > 0.f && c0 < __fadd_rn(ap, cl.bp0)) {
        float fh, fl;
        f_exact(a2.x, a2.y, cl.bh0, cl.bl0, c0, fh, fl);
        if (fh > 0.f) rs = fmaf(s0, fh, rs);
    }
    if (s1 > 0.f && c1 < __fadd_rn(ap, cl.bp1)) {
        float fh, fl;
        f_exact(a2.x, a2.y, cl.bh1, cl.bl1, c1, fh, fl);
        if (fh > 0.f) rs = fmaf(s1, fh, rs);
    }
    return rs;
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(FULLMASK, v, off);
    return v;
}

__device__ __forceinline__ bool unit_bit(const uint32_t* need, int words, int l, int jt)
{
    return (__ldg(need + (int64_t)l * words + (jt >> 5)) >> (jt & 31)) & 1u;
}

// Snapshot values of block (l, col) (written only for col < n).
__device__ __forceinline__ void put_snap(const EvalArgs& A, int l, int col, float zt, float ot)
{
    if (col < A.n) {
        const int64_t q = (int64_t)l * A.ntiles * TW + col;
        A.zt[q] = zt;
        A.ot[q] = ot;
    }
}

// Producer lane: registers the stage's transaction bytes on its full barrier
// and copies the stage's column constants and the (alpha hi, lo) pairs of rows
// [ra, ra + rows) -- as the 16-byte aligned superset [ra & ~1, (ra + rows + 1)
// & ~1) -- into the stage.  Returns the offset of row ra in arow[slot].
__device__ __forceinline__ int stage_side(const EvalArgs& A, Smem& S, int slot, int ra, int rows, uint32_t extra,
                                          int col)
{
    const uint32_t cb = SC * sizeof(float2) + SC * sizeof(float);
    int a0 = ra & ~1, a1 = (ra + rows + 1) & ~1;
    if (rows == 0) a0 = a1 = ra;
    const uint32_t ab = (uint32_t)(a1 - a0) * (uint32_t)sizeof(float2);
    mbar_expect(&S.full[slot], extra + ab + cb);
    bulk_copy(S.colB[slot], A.B2 + col, SC * sizeof(float2), &S.full[slot]);
    bulk_copy(S.colP[slot], A.Bp + col, SC * sizeof(float), &S.full[slot]);
    if (ab) bulk_copy(S.arow[slot], A.A2 + a0, ab, &S.full[slot]);
    return ra - a0;
}

// Barrier of the eight consumer warps on an mbarrier (bounded wait); phase
// counts the barriers this warp has passed.
__device__ __forceinline__ bool consumer_sync(Smem& S, uint32_t& phase)
{
    __syncwarp();
    if ((threadIdx.x & 31) == 0) mbar_arrive(&S.cbar);
    const bool ok = mbar_wait(&S.cbar, phase & 1u);
    phase++;
    return ok;
}

__device__ __forceinline__ void load_desc(const EvalArgs& A, int it, ItemDesc& d)
{
    const int4* src = reinterpret_cast<const int4*>(A.plan.desc + it);
    int4* dst = reinterpret_cast<int4*>(&d);
#pragma unroll
    for (int k = 0; k < (int)(sizeof(ItemDesc) / sizeof(int4)); k++) dst[k] = __ldg(src + k);
}

}  // namespace

// ================================================================= kernel
template <bool SNAP>
__global__ void __launch_bounds__(THREADS, 1) k_stream(const EvalArgs A, const __grid_constant__ TmaMaps T)
{
    extern __shared__ unsigned char smem_raw[];
    // TMA destinations must be 128-byte aligned: align the layout to 1 KB
    Smem& S = *reinterpret_cast<Smem*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < NSTAGES; s++) {
            mbar_init(&S.full[s], 1);
            mbar_init(&S.empty[s], CONSUMERS);
        }
        mbar_init(&S.cbar, CONSUMERS);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    // ------------------------------------------------------------ producer
    if (warp == CONSUMERS) {
        long long issued = 0;  // stages issued so far
        bool ok = true;
        auto next_slot = [&](int& slot) -> bool {
            slot = (int)(issued % NSTAGES);
            const long long use = issued / NSTAGES;
            return use == 0 || mbar_wait(&S.empty[slot], (uint32_t)((use - 1) & 1));
        };
        // the next item's index and descriptor are fetched one item ahead
        int nxt = 0;
        if (lane == 0) nxt = atomicAdd(A.work, 1);
        nxt = __shfl_sync(FULLMASK, nxt, 0);
        ItemDesc dn;
        bool act_n = true;
        if (nxt < A.nlist) {
            load_desc(A, nxt, dn);
            act_n = !A.unit_need || __ldg(A.item_active + dn.item);
        }
        for (;;) {
            const int it = nxt;
            if (it >= A.nlist) {
                int slot;
                if (!next_slot(slot)) { ok = false; break; }
                if (lane == 0) {
                    S.hdr[slot].flags = H_TERM;
                    mbar_arrive(&S.full[slot]);
                }
                issued++;
                break;
            }
            const ItemDesc d = dn;
            const bool act = act_n;
            if (lane == 0) nxt = atomicAdd(A.work, 1);
            nxt = __shfl_sync(FULLMASK, nxt, 0);
            if (nxt < A.nlist) {
                load_desc(A, nxt, dn);
                act_n = !A.unit_need || __ldg(A.item_active + dn.item);
            }
            if (!act) continue;
            for (int t = 0; t < d.nt && ok; t += 2) {
                const int jt = d.t0 + t;
                const int col = jt * TW;
                const bool two = t + 1 < d.nt;
                const bool tneed = d.kind == 0 || !A.unit_need || unit_bit(A.unit_need, A.unit_words, d.l, jt) ||
                                   (two && unit_bit(A.unit_need, A.unit_words, d.l, jt + 1));
                const int tst = tneed ? d.nst : 1;  // a skipped big tile pair sends one empty stage
                for (int si = 0; si < tst; si++) {
                    int slot;
                    if (!next_slot(slot)) { ok = false; break; }
                    float* dst = S.stage[slot];
                    // H_LAST marks every stage of the item's last tile pair (consumers
                    // read the flags of a pair's first stage)
                    int flags = (t == 0 && si == 0 ? H_FIRST : 0) | (t + 2 >= d.nt ? H_LAST : 0);
                    if (d.kind && d.nst <= NSTAGES) flags |= H_BIG_HELD;
                    if (d.kind && !tneed) flags |= H_SKIP;
                    int ra = d.r0, rows = d.rows;
                    uint32_t extra = 0;
                    if (d.kind == 0) {
                        if (!A.unit_need) {
                            extra = (uint32_t)rows * ROW_BYTES;
                        } else {
                            uint32_t cnt = 0;
                            for (int gi = d.pw[0] + lane; gi < d.pw[NWARPS]; gi += 32) {
                                const int4 g4 = __ldg(A.plan.pginfo + gi);
                                if (unit_bit(A.unit_need, A.unit_words, g4.x, jt) ||
                                    (two && unit_bit(A.unit_need, A.unit_words, g4.x, jt + 1)))
                                    cnt += (uint32_t)g4.z;
                            }
                            for (int off = 16; off >= 1; off >>= 1) cnt += __shfl_xor_sync(FULLMASK, cnt, off);
                            extra = cnt * ROW_BYTES;
                            if (cnt == 0) rows = 0;
                        }
                        if (t == 0) extra += (uint32_t)d.ngroups * 16u;
                    } else {
                        ra = d.r0 + si * STAGE_ROWS;
                        rows = tneed ? min(STAGE_ROWS, d.rows - si * STAGE_ROWS) : 0;
                        extra = (uint32_t)rows * ROW_BYTES;
                    }
                    if (lane == 0) {
                        const int a_sh = stage_side(A, S, slot, ra, rows, extra, col);
                        if (d.kind == 0 && t == 0)
                            bulk_copy(S.gstage[slot], A.plan.pginfo + d.pw[0], (uint32_t)d.ngroups * 16u,
                                      &S.full[slot]);
                        StageHdr& hh = S.hdr[slot];
                        hh.d = d;
                        hh.tile = jt; hh.sidx = si; hh.nst = tst; hh.flags = flags; hh.a_shift = a_sh;
                        if (d.kind == 0 && !A.unit_need) tma_rows(T, dst, col, d.r0, d.rows, &S.full[slot]);
                        if (d.kind == 1 && rows > 0) tma_rows(T, dst, col, ra, rows, &S.full[slot]);
                    }
                    if (d.kind == 0 && A.unit_need) {
                        __syncwarp();
                        for (int gi = d.pw[0] + lane; gi < d.pw[NWARPS]; gi += 32) {
                            const int4 g4 = __ldg(A.plan.pginfo + gi);
                            if (!(unit_bit(A.unit_need, A.unit_words, g4.x, jt) ||
                                  (two && unit_bit(A.unit_need, A.unit_words, g4.x, jt + 1))))
                                continue;
                            tma_rows(T, dst + (g4.y - d.r0) * SC, col, g4.y, g4.z, &S.full[slot]);
                        }
                    }
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&S.full[slot]);
                    issued++;
                }
            }
            if (!ok) break;
        }
        if (!ok) {
            if (lane == 0) atomicOr(A.err, 1);
            // wait (bounded) for the copies already issued into the ring
            for (long long k = (issued > NSTAGES ? issued - NSTAGES : 0); k < issued; k++)
                mbar_wait(&S.full[k % NSTAGES], (uint32_t)((k / NSTAGES) & 1));
        }
        return;
    }

    // ----------------------------------------------------------- consumers
    uint32_t cphase = 0;
#define CSYNC()                                    \
    do {                                           \
        if (!consumer_sync(S, cphase)) {           \
            if (lane == 0) atomicOr(A.err, 8);     \
            return;                                \
        }                                          \
    } while (0)
    long long consumed = 0;
    double psi_acc = 0.0;
    int gk0 = 0, gk1 = 0;  // small item: this warp's groups are ginfo[gk0, gk1)
    for (;;) {
        const int slot = (int)(consumed % NSTAGES);
        if (!mbar_wait(&S.full[slot], (uint32_t)((consumed / NSTAGES) & 1))) {
            if (lane == 0) atomicOr(A.err, 2);
            return;
        }
        const StageHdr& hs = S.hdr[slot];
        const int flags = hs.flags;
        if (flags & H_TERM) return;
        const int item = hs.d.item, jt = hs.tile, p = hs.d.p, kind = hs.d.kind;
        const int col0 = hs.d.col0, ncols = hs.d.ncols;
        const int64_t rbase = (int64_t)(((uint64_t)(uint32_t)hs.d.rb_hi << 32) | (uint32_t)hs.d.rb_lo);
        const int c0 = jt * TW + lane, c1 = c0 + TW;  // this lane's columns
        const bool two = jt + 1 < hs.d.t0 + hs.d.nt;
        const Col2 cl = load_cols(S, slot, lane);
        if (kind == 0) {
            // ---------------- small panel: a contiguous run of whole groups per warp
            const int rows = hs.d.rows;
            if (flags & H_FIRST) {
                const int ng = hs.d.ngroups;
                for (int k = threadIdx.x; k < ng; k += CONSUMERS * 32) S.ginfo[k] = S.gstage[slot][k];
                for (int i = threadIdx.x; i < rows; i += CONSUMERS * 32) S.rowacc[i] = 0.f;
                gk0 = hs.d.pw[warp] - hs.d.pw[0];
                gk1 = hs.d.pw[warp + 1] - hs.d.pw[0];
                psi_acc = 0.0;
                CSYNC();
            }
            const float* st = S.stage[slot];
            const float2* ar = S.arow[slot] + hs.a_shift;
            float cacc0 = 0.f, cacc1 = 0.f;
            for (int k = gk0; k < gk1; k++) {
                const int4 gi4 = S.ginfo[k];
                const int l = gi4.x, g = gi4.z, sr = gi4.w;
                if (A.unit_need && !(unit_bit(A.unit_need, A.unit_words, l, jt) ||
                                     (two && unit_bit(A.unit_need, A.unit_words, l, jt + 1))))
                    continue;
                Acc a0 = {0.f, 0.f, 0.f, 0.f}, a1 = {0.f, 0.f, 0.f, 0.f};
                float O0 = 0.f, O1 = 0.f;
                bool any = false;
#pragma unroll 2
                for (int r = sr; r < sr + g; r++)
                    any |= row_a<SNAP>(ar[r], st[r * SC + lane], st[r * SC + lane + 32], cl, a0, a1, O0, O1);
                float s0 = 0.f, s1 = 0.f;
                if (__any_sync(FULLMASK, any)) {
                    double p0, p1;
                    s0 = block_scale(a0.Sh, a0.Sl, A, p0);
                    s1 = block_scale(a1.Sh, a1.Sl, A, p1);
                    psi_acc += p0 + p1;
                    cacc0 = fmaf(s0, __fadd_rn(a0.Ph, a0.Pl), cacc0);
                    cacc1 = fmaf(s1, __fadd_rn(a1.Ph, a1.Pl), cacc1);
                }
                if (SNAP) {
                    put_snap(A, l, c0, z_up(a0.Sh, a0.Sl), __fsqrt_ru(O0));
                    if (two) put_snap(A, l, c1, z_up(a1.Sh, a1.Sl), __fsqrt_ru(O1));
                }
                if (__any_sync(FULLMASK, s0 > 0.f || s1 > 0.f)) {
                    for (int r = sr; r < sr + g; r++) {
                        const float rs = warp_sum(row_b(ar[r], st[r * SC + lane], st[r * SC + lane + 32], cl, s0, s1));
                        if (lane == 0) S.rowacc[r] += rs;
                    }
                }
            }
            S.colacc[warp][jt * TW - col0 + lane] = cacc0;
            S.colacc[warp][jt * TW - col0 + lane + TW] = cacc1;
            __syncwarp();
            if (lane == 0) mbar_arrive(&S.empty[slot]);
            consumed++;
            if (flags & H_LAST) {
#pragma unroll
                for (int off = 16; off >= 1; off >>= 1) psi_acc += __shfl_xor_sync(FULLMASK, psi_acc, off);
                if (lane == 0) S.psi_w[warp] = psi_acc;
                CSYNC();
                const int tid = threadIdx.x;
                for (int i = tid; i < rows; i += CONSUMERS * 32) A.rowpart[rbase + i] = (double)S.rowacc[i];
                for (int c = tid; c < ncols; c += CONSUMERS * 32) {
                    double v = 0.0;
#pragma unroll
                    for (int w = 0; w < CONSUMERS; w++) v += (double)S.colacc[w][c];
                    A.colpart[(int64_t)p * A.n + col0 + c] = v;
                }
                if (tid == 0) {
                    double v = 0.0;
                    for (int w = 0; w < CONSUMERS; w++) v += S.psi_w[w];
                    A.psipart[item] = v;
                }
                CSYNC();
            }
            continue;
        }
        // ---------------- big group: this tile pair spans nst stages
        const int l = hs.d.l, r0 = hs.d.r0, g = hs.d.rows;
        const int nst = hs.nst;
        const bool held = (flags & H_BIG_HELD) != 0;
        const bool need = !(flags & H_SKIP);
        const bool racc_smem = g <= BIG_SMEM_ROWS;
        double* racc_g = A.rowpart + rbase;
        const int wr0 = warp * WROWS;  // this warp's rows of each stage: [wr0, wr0 + WROWS)
        if (flags & H_FIRST) {
            for (int sb = 0; sb < g; sb += STAGE_ROWS)
                if (lane < WROWS) {
                    const int R = sb + wr0 + lane;
                    if (R < g) {
                        if (racc_smem) S.rowacc[R] = 0.f;
                        else racc_g[R] = 0.0;
                    }
                }
            psi_acc = 0.0;
            __syncwarp();
        }
        Acc a0 = {0.f, 0.f, 0.f, 0.f}, a1 = {0.f, 0.f, 0.f, 0.f};
        float O0 = 0.f, O1 = 0.f;
        bool any = false;
        const long long pair_first = consumed;  // stage index of this pair's first stage
        if (need) {
            for (int si = 0; si < nst; si++) {
                const int sl = (int)(consumed % NSTAGES);
                if (si > 0 && !mbar_wait(&S.full[sl], (uint32_t)((consumed / NSTAGES) & 1))) {
                    if (lane == 0) atomicOr(A.err, 4);
                    return;
                }
                const float* st = S.stage[sl];
                const float2* ar = S.arow[sl] + S.hdr[sl].a_shift;
                const int rows = min(STAGE_ROWS, g - si * STAGE_ROWS);
                const int rend = min(wr0 + WROWS, rows);
#pragma unroll 2
                for (int r = wr0; r < rend; r++)
                    any |= row_a<SNAP>(ar[r], st[r * SC + lane], st[r * SC + lane + 32], cl, a0, a1, O0, O1);
                if (!held) {
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&S.empty[sl]);
                }
                consumed++;
            }
        } else {
            __syncwarp();
            if (lane == 0) mbar_arrive(&S.empty[slot]);
            consumed++;
        }
        S.red[warp][lane] = make_float4(a0.Sh, a0.Sl, a0.Ph, a0.Pl);
        S.red[warp][lane + 32] = make_float4(a1.Sh, a1.Sl, a1.Ph, a1.Pl);
        if (SNAP) {
            S.redO[warp][lane] = O0;
            S.redO[warp][lane + 32] = O1;
        }
        const bool wany = __any_sync(FULLMASK, any);
        if (lane == 0) S.anyw[warp] = wany ? 1 : 0;
        CSYNC();
        bool cany = false;
#pragma unroll
        for (int w = 0; w < CONSUMERS; w++) cany |= S.anyw[w] != 0;
        // every warp combines the partials of its two columns in warp order
        float s[2] = {0.f, 0.f};
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int c = lane + h * TW, col = jt * TW + c;
            float zt = 0.f, ot = 0.f;
            if (SNAP) {
                float o = S.redO[0][c];
                for (int w = 1; w < CONSUMERS; w++) o += S.redO[w][c];
                ot = __fsqrt_ru(o);
            }
            float sc = 0.f, pp = 0.f;
            if (cany) {
                const float4 v = S.red[0][c];
                float hh = v.x, hl = v.y, ph = v.z, pl = v.w;
                for (int w = 1; w < CONSUMERS; w++) {
                    const float4 u = S.red[w][c];
                    df_add(hh, hl, u.x, u.y);
                    df_add(ph, pl, u.z, u.w);
                }
                double psi;
                sc = block_scale(hh, hl, A, psi);
                if (warp == 0) psi_acc += psi;
                zt = z_up(hh, hl);
                pp = __fadd_rn(ph, pl);
            }
            s[h] = sc;
            if (warp == 0 && (h == 0 || two) && col < A.n) {
                A.colpart[(int64_t)p * A.n + col] = (double)__fmul_rn(sc, pp);
                if (SNAP && need) put_snap(A, l, col, zt, ot);
            }
        }
        CSYNC();  // red / anyw free for the next pair
        if (__any_sync(FULLMASK, s[0] > 0.f || s[1] > 0.f)) {
            for (int si = 0; si < nst; si++) {
                const int rows = min(STAGE_ROWS, g - si * STAGE_ROWS);
                const int rend = min(wr0 + WROWS, rows);
                if (held) {
                    const int hsl = (int)((pair_first + si) % NSTAGES);
                    const float* st = S.stage[hsl];
                    const float2* ar = S.arow[hsl] + S.hdr[hsl].a_shift;
                    for (int r = wr0; r < rend; r++) {
                        const float rs = warp_sum(row_b(ar[r], st[r * SC + lane], st[r * SC + lane + 32], cl, s[0], s[1]));
                        if (lane == 0) {
                            const int R = si * STAGE_ROWS + r;
                            if (racc_smem) S.rowacc[R] += rs;
                            else racc_g[R] += (double)rs;
                        }
                    }
                } else {
                    // the stage has left the ring: re-read its rows from L2
                    for (int r = wr0; r < rend; r++) {
                        const int R = si * STAGE_ROWS + r;
                        const float* rowp = A.C + (int64_t)(r0 + R) * A.ldc;
                        const float x0 = c0 < A.n ? __ldg(rowp + c0) : 0.f;
                        const float x1 = c1 < A.n ? __ldg(rowp + c1) : 0.f;
                        const float rs = warp_sum(row_b(__ldg(A.A2 + r0 + R), x0, x1, cl, s[0], s[1]));
                        if (lane == 0) {
                            if (racc_smem) S.rowacc[R] += rs;
                            else racc_g[R] += (double)rs;
                        }
                    }
                }
            }
        }
        if (held && need) {
            __syncwarp();
            if (lane == 0)
                for (int si = 0; si < nst; si++) mbar_arrive(&S.empty[(int)((pair_first + si) % NSTAGES)]);
        }
        if (flags & H_LAST) {
            if (warp == 0) {
#pragma unroll
                for (int off = 16; off >= 1; off >>= 1) psi_acc += __shfl_xor_sync(FULLMASK, psi_acc, off);
                if (lane == 0) A.psipart[item] = psi_acc;
            }
            CSYNC();
            if (racc_smem)
                for (int i = threadIdx.x; i < g; i += CONSUMERS * 32) A.rowpart[rbase + i] = (double)S.rowacc[i];
            CSYNC();
        }
    }
}

#undef CSYNC

size_t stream_smem_bytes() { return sizeof(Smem) + 1024; }

void launch_stream(const EvalArgs& a, const TmaMaps& T, int n_ctas, cudaStream_t st)
{
    const int sm = (int)stream_smem_bytes();
    if (a.zt) {
        cudaFuncSetAttribute(k_stream<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        k_stream<true><<<n_ctas, THREADS, sm, st>>>(a, T);
    } else {
        cudaFuncSetAttribute(k_stream<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        k_stream<false><<<n_ctas, THREADS, sm, st>>>(a, T);
    }
}

// ------------------------------------------------------------ TMA maps
namespace {
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}
}  // namespace

std::string make_tmaps(const float* C, int64_t ldc, int64_t m, int64_t n, TmaMaps& T)
{
    EncodeTiledFn enc = encode_fn();
    if (!enc) return "cuTensorMapEncodeTiled is unavailable";
    const cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)m};
    const cuuint64_t strides[1] = {(cuuint64_t)ldc * sizeof(float)};
    const cuuint32_t estr[2] = {1, 1};
    for (int k = 0; k < TMA_BOXES; k++) {
        const cuuint32_t box[2] = {(cuuint32_t)SC, 1u << k};
        CUresult r = enc(&T.box[k], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(C), dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return "cuTensorMapEncodeTiled failed with code " + std::to_string((int)r);
    }
    return "";
}

}  // namespace otgs
