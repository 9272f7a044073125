// otgs_stream.cu -- the evaluation of the dual (Eq. 4) and its gradient
// (Eq. 5): one pass over C that bounds every block, then the exact sums of
// the blocks the bound does not rule out.
//
// k_stream, persistent, CTAS_PER_SM CTAs per SM, warp-specialised:
//  * a producer warp takes work items (a panel of whole groups x ITEM_COLS
//    columns; host-built descriptors fetched three items ahead) from a global
//    counter and streams each item's rows, STAGE_ROWS at a time, into a ring
//    of NSTAGES shared-memory stages: the rows of C as 2D TMA boxes (1 KB per
//    row), the rows' alpha records and (group, end) records as bulk copies,
//    and on an item's first stage its columns' beta constants.  Stages
//    complete on mbarrier transaction counts;
//  * NWARPS consumer warps: warp w owns the item's columns [32 w, 32 w + 32),
//    one per lane, and walks every row of every stage.  For each element the
//    lane forms y = fl(fl(A'_i - c_ij) + B'_j) (A', B' alpha, beta rounded up,
//    so y >= f_ij where f_ij > 0) and adds [y]_+^2 to its block's FP32 sum S',
//    an upper bound of z^2 = ||[f_[l]]_+||^2 within a stated relative error.
//    4-row chunks where no y can be positive (the max over the chunk) are
//    skipped, and so are groups with no such chunk.  At a block's last row
//    a bound at or below theta^2 (with its error) means s = 0 (Eq. 5): the
//    block adds nothing.  The other ("flagged") blocks of a 32-column tile
//    are recorded for the exact-sum kernel.  The work per element is the same
//    in every lane and warp whatever the iterate.  Pieces of a split group
//    store their partial bound sums; the split-finish kernel adds them.  A
//    snapshot evaluation also needs z~ (an upper bound: the bound itself) and
//    o~ (Def. 1-2) of every block, so it walks every group.
//
// k_exact, k_exact_tall: the flagged blocks.  f is formed in double-float
// with TwoSum, S = sum [f]_+^2 and P = sum [f]_+ are summed in a fixed
// order, Eq. 5 gives the shrink s and psi, and a second sweep adds t_ij =
// s [f_ij]_+ into the row sums.  Row and column sums and psi are int64 fixed
// point (atomic adds whose total does not depend on their order), so the
// results are deterministic, and a screened evaluation (skipped blocks
// contribute exact zeros) equals a dense one bit for bit.
//
// Every wait is on an mbarrier and gives up after WAIT_NS; on timeout the
// kernel records an error in A.err, the producer waits (bounded) for the
// copies it issued, and all warps return.
#include <mutex>
#include <string>

#include "otgs_internal.cuh"

namespace otgs {

#define FULLMASK 0xffffffffu

namespace {

constexpr int CONSUMERS = NWARPS;
constexpr int THREADS = (CONSUMERS + 1) * 32;
constexpr int IC = ITEM_COLS;                          // columns of a stage row
constexpr int SR = STAGE_ROWS;                         // rows of a stage
constexpr uint32_t ROW_BYTES = IC * 4;                 // a TMA box row, zero-filled past column n
constexpr unsigned long long WAIT_NS = 2000000000ull;  // give up a wait after 2 s
constexpr int DESC_WORDS = (int)(sizeof(ItemDesc) / sizeof(int));
static_assert(DESC_WORDS <= 32, "a descriptor is spread over the producer's lanes");
static_assert(SR == 32, "the producer maps one lane to each row of a stage");


enum : int { H_FIRST = 1, H_TERM = 4 };

// What the consumers need about a stage, written by the producer.
struct StageHdr {
    ItemDesc d;
    int ra;       // the stage's first sorted row
    int nr;       // its rows (<= SR)
    int flags;
    int tiled;    // 0: rows of ITEM_COLS ([row][IC]); 1: per warp tile ([warp][row][TW])
};

struct Smem {
    float stage[NSTAGES][SR * IC];   // NSTAGES x 32 KB; see StageHdr::tiled
    float4 rowA[NSTAGES][SR];        // (alpha hi, alpha lo, A', 0) of the stage's rows
    int4 rowG[NSTAGES][SR];          // (group, first row, end row, 0) of the stage's rows
    float2 colB[NSTAGES][IC];        // item's first stage: (beta hi, lo) of its columns
    uint32_t rmaskw[NSTAGES][CONSUMERS];  // screened: bit r set = warp w evaluates row r's block
    StageHdr hdr[NSTAGES];
    uint64_t full[NSTAGES];
    uint64_t empty[NSTAGES];
};
static_assert(CTAS_PER_SM * (sizeof(Smem) + 2048) <= 228 * 1024, "shared memory of the CTAs of one SM");

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

// Wait for the phase with the given parity to complete; false after limit ns.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, unsigned long long limit)
{
    if (mbar_try(b, parity)) return true;
    const unsigned long long t0 = gtime();
    for (;;) {
        for (int i = 0; i < 64; i++)
            if (mbar_try(b, parity)) return true;
        if (gtime() - t0 > limit) return false;
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

// One TMA box: rows [y, y + 2^k) x columns [x, x + IC) of C into dst.
__device__ __forceinline__ void tma_box(const CUtensorMap* M, int k, float* dst, int x, int y, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(su32(dst)),
        "l"(reinterpret_cast<uint64_t>(M + k)), "r"(x), "r"(y), "r"(su32(bar))
        : "memory");
}

// Orders this thread's later tensor copies after the descriptor's contents
// (written to global memory before the launch).
__device__ __forceinline__ void tmap_acquire(const CUtensorMap* M)
{
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(M))
                 : "memory");
}

// Rows [y, y + rows) (rows <= STAGE_ROWS) into dst rows [0, rows): one box per
// set bit of rows, so exactly the requested rows are read.
__device__ __forceinline__ void tma_rows(const CUtensorMap* M, float* dst, int x, int y, int rows, uint64_t* bar)
{
    int off = 0;
#pragma unroll
    for (int k = TMA_BOXES - 1; k >= 0; k--)
        if (rows & (1 << k)) {
            tma_box(M, k, dst + off * IC, x, y + off, bar);
            off += 1 << k;
        }
}

// The same for one 32-column tile: rows of TW floats at dst + r * TW.
__device__ __forceinline__ void tma_tile_rows(const CUtensorMap* M, float* dst, int x, int y, int rows, uint64_t* bar)
{
    int off = 0;
#pragma unroll
    for (int k = TMA_BOXES - 1; k >= 0; k--)
        if (rows & (1 << k)) {
            asm volatile(
                "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
                "[%4];" ::"r"(su32(dst + off * TW)),
                "l"(reinterpret_cast<uint64_t>(M + TMA_BOXES + k)), "r"(x), "r"(y + off), "r"(su32(bar))
                : "memory");
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

// (h, l) += (oh, ol)
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

// (h, l) = (ah + al) * (bh + bl) to ~2^-46 relative.
__device__ __forceinline__ void df_mul(float ah, float al, float bh, float bl, float& h, float& l)
{
    h = __fmul_rn(ah, bh);
    l = fmaf(ah, bh, -h);
    l = fmaf(ah, bl, fmaf(al, bh, l));
}

// Eq. 5 for one block from S = ||[f_[l]]_+||^2: the shrink factor
// s = [z - theta]_+ / (gamma z) and psi = [z - theta]_+^2 / (2 gamma) as a
// float pair (psh, psl).  FP32 only: GB300's FP64 rate is a small fraction
// of its FP32 rate, and this runs once per block.
__device__ __forceinline__ float block_scale(float Sh, float Sl, const EvalArgs& A, float& psh, float& psl)
{
    psh = 0.f;
    psl = 0.f;
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
    float qh, ql;
    df_mul(dh, dl, dh, dl, qh, ql);
    df_mul(qh, ql, A.inv2g_hi, A.inv2g_lo, psh, psl);
    return __fdiv_rn(ds, __fmul_rn(A.gamma, __fadd_rn(zh, zl)));
}

// z rounded up (snapshot value z~ of Def. 1, kept as an upper bound).
__device__ __forceinline__ float z_up(float Sh, float Sl) { return __fsqrt_ru(fmaxf(__fadd_ru(Sh, Sl), 0.f)); }

// The cheap test of one element: false only when f_ij is certainly <= 0.
__device__ __forceinline__ bool maybe_pos(float ap, float c, float bp)
{
    return __fadd_rn(__fsub_rn(ap, c), bp) > 0.f;
}

// Whether a block may have s > 0 (Eq. 5), from the FP32 bound S' = sum of
// [y]_+^2 over its rows (y as bound_up describes, [y]_+ >= [f]_+ for every
// element): S' summed by k fused multiply-adds and additions of non-negative
// terms is at least (1 - 2^-24)^k of the exact sum, so ||[f]_+||^2 <= S' (1 +
// (k + 4) 2^-23) holds, and a block at or below thr_flag = RD(theta^2 (1 -
// 2^-21)) has z < theta by far more than the exact sums' rounding: its s is 0.
// k counts the rows and the partial sums added.  theta = 0: every block with
// some [y]_+ > 0.
__device__ __forceinline__ float sp_bound(float Sp, int k) { return fmaf(Sp, (float)(k + 4) * 0x1p-23f, Sp); }
__device__ __forceinline__ bool flag_block(float Sp, int k, float thr) { return sp_bound(Sp, k) > thr; }
// The same bound rounded up, as a snapshot value z~ >= z (Def. 1).
__device__ __forceinline__ float sp_up(float Sp, int k)
{
    return __fsqrt_ru(__fmaf_ru(Sp, __fmul_ru((float)(k + 4), 0x1p-23f), Sp));
}

// One element of the stream's pass: y = fl(fl(A' - c) + B') (>= f where
// f > 0); S' += [y]_+^2, and for a snapshot the sum of [y]_-^2.
template <bool SNAP>
__device__ __forceinline__ void elem_pass(float ap, float c, float bp, float& Sp, float& O)
{
    const float y = __fadd_rn(__fsub_rn(ap, c), bp);
    const float p = fmaxf(y, 0.f);  // a NaN y counts as 0
    Sp = fmaf(p, p, Sp);
    if (SNAP) {
        const float q = fminf(y, 0.f);
        O = fmaf(q, q, O);
    }
}

// Bit q set: chunk q (rows [4q, 4q + 4)) of the stage may hold an f > 0 in
// this lane's column.  Rows past the stage's end hold stale data and are
// masked by the caller.
template <int RS>
__device__ __forceinline__ uint32_t chunk_marks(const float* st, const float4* rA, float bp)
{
    uint32_t cm = 0u;
#pragma unroll
    for (int q = 0; q < SR / 4; q++) {
        const int r = 4 * q;
        const float x0 = __fsub_rn(rA[r + 0].z, st[(r + 0) * RS]);
        const float x1 = __fsub_rn(rA[r + 1].z, st[(r + 1) * RS]);
        const float x2 = __fsub_rn(rA[r + 2].z, st[(r + 2) * RS]);
        const float x3 = __fsub_rn(rA[r + 3].z, st[(r + 3) * RS]);
        const float mx = fmaxf(fmaxf(x0, x1), fmaxf(x2, x3));  // a NaN operand yields the other one
        if (__fadd_rn(mx, bp) > 0.f) cm |= 1u << q;
    }
    return cm;
}

// Chunks that overlap rows [s, e) (s < e).
__device__ __forceinline__ uint32_t chunks_in(int s, int e)
{
    return ((2u << ((e - 1) >> 2)) - 1u) & ~((1u << (s >> 2)) - 1u);
}

// Chunks with at least one row set in a 32-row mask.
__device__ __forceinline__ uint32_t chunks_of_rows(uint32_t rows)
{
    uint32_t c = 0u;
#pragma unroll
    for (int q = 0; q < SR / 4; q++)
        if ((rows >> (4 * q)) & 0xfu) c |= 1u << q;
    return c;
}

// t_ij = s f_ij (FP32) on the fixed-point grid: t * 2^k is exact in FP32
// (below 2^61 by the choice of k), so this is the integer nearest to t 2^k.
// The integer nearest to x (ties to even) for |x| < 2^63, with 32-bit
// conversions only (a 64-bit one runs on GB300's narrow FP64 pipe): x =
// h 2^32 + r with h = floor(|x| 2^-32) and r = |x| - h 2^32 both exact in FP32
// (r holds the low bits of |x|'s 24-bit significand).
__device__ __forceinline__ long long f2ll_rn(float x)
{
    const float ax = fabsf(x);
    const float h = floorf(__fmul_rn(ax, 0x1p-32f));
    const float r = fmaf(-h, 0x1p32f, ax);
    const long long q = ((long long)__float2int_rz(h) << 32) + (long long)__float2uint_rn(r);
    return x < 0.f ? -q : q;
}

__device__ __forceinline__ unsigned long long t_q(float t, float to_fx)
{
    return (unsigned long long)f2ll_rn(__fmul_rn(t, to_fx));
}

// A block's column-sum term s P (P = Ph + Pl) in fixed point: s P as a float
// pair, each part rounded to the grid (an error below one grid step).
__device__ __forceinline__ long long col_q(float s, float Ph, float Pl, float to_fx)
{
    const float ph = __fmul_rn(s, Ph);
    const float pl = fmaf(s, Pl, fmaf(s, Ph, -ph));
    return f2ll_rn(__fmul_rn(ph, to_fx)) + f2ll_rn(__fmul_rn(pl, to_fx));
}

// Snapshot values of block (l, col) (written only for a real column).
__device__ __forceinline__ void put_snap(const EvalArgs& A, int l, int col, bool real, float zt, float ot)
{
    if (real) {
        const int64_t q = (int64_t)l * A.ntiles * TW + col;
        A.zt[q] = zt;
        A.ot[q] = ot;
    }
}

// The block of this lane's column that is being accumulated.
struct Block {
    int gl, gstart, gend;  // group and the sorted rows [gstart, gend) summed in this item
    bool split;            // a piece of a group cut over several items
    bool need;             // evaluated by this warp (always, unless screened)
    float Sp;              // FP32 bound sum of [y]_+^2
    float O;               // sum of [y]_-^2 (snapshot evaluations)
};

// Per-lane constants of the current item and the stage being consumed.
struct Ctx {
    const float* st;   // stage, offset to this lane's column
    int rs;            // the stage's row stride (floats)
    const float4* rA;  // stage's alpha records
    int ra, nr;        // first sorted row of the stage, rows in it
    float bp;          // B' of this lane's column (-inf past the problem's last column)
    int colg;          // this lane's column in the concatenation of the problems' columns
    bool real;         // the lane's column exists (the item's last chunk may be narrower)
    uint32_t U;        // chunks of the stage marked by some lane (dense path)
    int r0;            // first sorted row of the item
    int rend;          // end row of the item
    int pslot;         // a piece of a split group: its partial-sum slot
    int prob;          // the item's problem
};

__device__ __forceinline__ void open_block(Block& b, const int4& g, bool need, const Ctx& x)
{
    b.gl = g.x;
    b.split = g.y < x.r0 || g.z > x.rend;  // a group cut into pieces: this item sums one
    b.gstart = max(g.y, x.r0);
    b.gend = min(g.z, x.rend);
    b.need = need;
    b.Sp = 0.f;
    b.O = 0.f;
}

// The block is complete: flagged (its FP32 bound does not rule out z > theta)
// it goes to the exact-sum kernel, which finishes it; otherwise its s is 0
// and it adds nothing.  A snapshot stores the bound as z~ (the exact-sum
// kernel replaces it for the flagged blocks) and o~.  A piece of a split
// group only stores its partial sums; the split-finish kernel adds the
// pieces in order and decides.
template <bool SNAP>
__device__ __forceinline__ void finish_block(const EvalArgs& A, const Block& b, const Ctx& x, int lane)
{
    if (b.split) {
        float* q = A.split_part + ((int64_t)x.pslot * ITEM_COLS + (threadIdx.x >> 5) * TW + lane) * SPLIT_VALS;
        q[0] = b.Sp;
        q[1] = b.O;
        return;
    }
    const int k = b.gend - b.gstart;
    const uint32_t fw = __ballot_sync(FULLMASK, x.real && flag_block(b.Sp, k, A.thr_flag));
    if (fw) add_xentry(A, b.gstart, b.gend, x.colg - lane, x.prob, b.gl, fw, lane);
    if (SNAP) put_snap(A, b.gl, x.colg, x.real, sp_up(b.Sp, k), __fsqrt_ru(b.O));
}

// Dense path: the marked chunks of rows [s, e) of the block's group.
__device__ __forceinline__ void block_marked_rows(Block& b, const Ctx& x, int s, int e)
{
    uint32_t qm = x.U & chunks_in(s, e);
    float O = 0.f;
    while (qm) {
        const int q = __ffs(qm) - 1;
        qm &= qm - 1u;
        const int r0 = max(4 * q, s), r1 = min(4 * q + 4, e);
        if (r0 == 4 * q && r1 == 4 * q + 4) {
            const float c0 = x.st[(r0 + 0) * x.rs], c1 = x.st[(r0 + 1) * x.rs], c2 = x.st[(r0 + 2) * x.rs],
                        c3 = x.st[(r0 + 3) * x.rs];
            elem_pass<false>(x.rA[r0 + 0].z, c0, x.bp, b.Sp, O);
            elem_pass<false>(x.rA[r0 + 1].z, c1, x.bp, b.Sp, O);
            elem_pass<false>(x.rA[r0 + 2].z, c2, x.bp, b.Sp, O);
            elem_pass<false>(x.rA[r0 + 3].z, c3, x.bp, b.Sp, O);
        } else {
            for (int r = r0; r < r1; r++) elem_pass<false>(x.rA[r].z, x.st[r * x.rs], x.bp, b.Sp, O);
        }
    }
}

// Snapshot path: every row of [r, e).
__device__ __forceinline__ void scan_rows(Block& b, const Ctx& x, int r, int e)
{
    for (; r + 4 <= e; r += 4) {
        const float c0 = x.st[(r + 0) * x.rs], c1 = x.st[(r + 1) * x.rs], c2 = x.st[(r + 2) * x.rs],
                    c3 = x.st[(r + 3) * x.rs];
        elem_pass<true>(x.rA[r + 0].z, c0, x.bp, b.Sp, b.O);
        elem_pass<true>(x.rA[r + 1].z, c1, x.bp, b.Sp, b.O);
        elem_pass<true>(x.rA[r + 2].z, c2, x.bp, b.Sp, b.O);
        elem_pass<true>(x.rA[r + 3].z, c3, x.bp, b.Sp, b.O);
    }
    for (; r < e; r++) elem_pass<true>(x.rA[r].z, x.st[r * x.rs], x.bp, b.Sp, b.O);
}

}  // namespace

// ================================================================= kernel
template <bool SNAP>
__global__ void __launch_bounds__(THREADS, CTAS_PER_SM) k_stream(const __grid_constant__ EvalArgs A)
{
    if (A.gate && !*A.gate) return;  // a skipped solver trial
    if (A.ctl->wl) return;           // screened, and the screen's block sets are the work
    extern __shared__ unsigned char smem_raw[];
    // TMA destinations must be 128-byte aligned: align the layout to 1 KB
    Smem& S = *reinterpret_cast<Smem*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < NSTAGES; s++) {
            mbar_init(&S.full[s], 1);
            mbar_init(&S.empty[s], CONSUMERS);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    const unsigned long long wlim = A.wait_ns ? A.wait_ns : WAIT_NS;  // limit of the ring's waits

    // ------------------------------------------------------------ producer
    if (warp == CONSUMERS) {
        const bool screened = A.unit_need != nullptr;
        long long issued = 0;  // stages issued so far
        unsigned long long cstreamed = 0;  // bytes of C requested (lane 0)
        bool ok = true;
        auto next_slot = [&](int& slot) -> bool {
            slot = (int)(issued % NSTAGES);
            const long long use = issued / NSTAGES;
            return use == 0 || mbar_wait(&S.empty[slot], (uint32_t)((use - 1) & 1), wlim);
        };
        // Items flow through a software pipeline so that no load is waited on
        // right after it is issued: at the start of item k the counter is bumped
        // for item k+3, the descriptor of item k+2 is loaded (lane w holds word
        // w) and the active flag of item k+1.
        auto fetch = [&]() -> int { return lane == 0 ? atomicAdd(&A.ctl->work, 1) : 0; };
        auto bcast = [&](int v) -> int { return __shfl_sync(FULLMASK, v, 0); };
        auto load_w = [&](int idx) -> int {
            return (idx < A.nlist && lane < DESC_WORDS) ? __ldg(reinterpret_cast<const int*>(A.desc + idx) + lane) : 0;
        };
        auto load_act = [&](int idx, int w) -> int {
            const int item = __shfl_sync(FULLMASK, w, 0), prob = __shfl_sync(FULLMASK, w, 11);
            if (idx >= A.nlist) return 0;
            int act = 1;  // lane 0's value is the one used
            if (A.item_active && lane == 0) act = (int)__ldg(A.item_active + item);
            if (A.prob_active && lane == 0 && !__ldg(A.prob_active + prob)) act = 0;
            return act;
        };
        // lane k: the item's stage boundary k (first rows, then the end), 32 at a time
        auto load_st = [&](int idx, int w, int base) -> int {
            const int st0 = __shfl_sync(FULLMASK, w, 12), nst = __shfl_sync(FULLMASK, w, 6);
            return (idx < A.nlist && base + lane <= nst) ? __ldg(A.stage_row0 + st0 + base + lane) : 0;
        };
        int fenced = -1;  // the problem whose tensor maps were last acquired
        int i0 = bcast(fetch());
        int w0 = load_w(i0);
        int a0 = load_act(i0, w0);

        int v0 = load_st(i0, w0, 0);
        int i1 = bcast(fetch());
        int w1 = load_w(i1);
        int i2r = fetch();
        for (;;) {
            if (i0 >= A.nlist) {
                int slot;
                if (!next_slot(slot)) { ok = false; break; }
                if (lane == 0) {
                    S.hdr[slot].flags = H_TERM;
                    mbar_arrive(&S.full[slot]);
                }
                issued++;
                break;
            }
            const int a1 = load_act(i1, w1);
            const int v1 = load_st(i1, w1, 0);
            const int i2 = bcast(i2r);
            const int w2 = load_w(i2);
            const int i3r = fetch();
            if (bcast(a0)) {
                const int col0 = __shfl_sync(FULLMASK, w0, 4), nst = __shfl_sync(FULLMASK, w0, 6);
                const int sbase = __shfl_sync(FULLMASK, w0, 7);
                const int prob = __shfl_sync(FULLMASK, w0, 11);
                const ProbDesc pd = A.inline_maps ? A.pd0 : A.probs[prob];
                const CUtensorMap* maps =
                    A.inline_maps ? &A.tm0.box[0] : A.maps + (int64_t)prob * 2 * TMA_BOXES;
                if (!A.inline_maps && prob != fenced) {  // descriptors in global memory: acquire them for the tensor proxy
                    if (lane == 0)
                        for (int k = 0; k < TMA_BOXES; k++) tmap_acquire(maps + k);
                    if (lane < CONSUMERS)
                        for (int k = 0; k < TMA_BOXES; k++) tmap_acquire(maps + TMA_BOXES + k);
                    fenced = prob;
                }
                // screened: the stages with a needed row (one bit per stage, read a
                // word at a time), and this lane's row's needed tiles for the next
                // such stage, loaded one needed stage ahead
                int need_wi = -1;
                uint32_t need_w = 0u;
                auto next_on = [&](int s0) -> int {
                    for (int q = s0; q < nst; q++) {
                        const int gs = sbase + q;
                        if ((gs >> 5) != need_wi) {
                            need_wi = gs >> 5;
                            need_w = __ldg(A.stage_need + need_wi);
                        }
                        if ((need_w >> (gs & 31)) & 1u) return q;
                    }
                    return nst;
                };
                int snext = screened ? next_on(0) : 0;
                uint32_t m8n = (screened && snext < nst) ? (uint32_t)__ldg(A.stage_m8 + (int64_t)(sbase + snext) * SR + lane)
                                                        : 0xffu;
                bool first = true;  // no stage of this item issued yet
                int wb = 0;         // first stage boundary held in v0
                for (int s = 0; s < nst; s++) {
                    if (s - wb >= 31) {  // a long item: the next 32 boundaries
                        wb = s;
                        v0 = load_st(i0, w0, wb);
                    }
                    if (screened && s != snext) continue;  // no row of this stage is needed: not sent
                    const int ra = __shfl_sync(FULLMASK, v0, s - wb);
                    const int nr = __shfl_sync(FULLMASK, v0, s - wb + 1) - ra;
                    uint32_t m8 = 0xffu;  // this lane's row: bit w = warp w evaluates its block
                    uint32_t need = nr == 32 ? FULLMASK : ((1u << nr) - 1u);
                    if (screened) {
                        m8 = m8n;
                        snext = next_on(s + 1);
                        if (snext < nst) m8n = __ldg(A.stage_m8 + (int64_t)(sbase + snext) * SR + lane);
                        need = __ballot_sync(FULLMASK, m8 != 0u);
                        if (!need) continue;  // (not reached: the stage's bit says some row is needed)
                    }
                    uint32_t wmask = 0u;   // lane w < CONSUMERS: rows evaluated by warp w (screened)
                    uint32_t tiles = 0u;
                    bool tiled = false;
                    if (screened) {
#pragma unroll
                        for (int w = 0; w < CONSUMERS; w++) {
                            const uint32_t bw = __ballot_sync(FULLMASK, (m8 >> w) & 1u);
                            if (lane == w) wmask = bw;
                        }
                        // When the needed (row, tile) pairs are sparse, load per 32-column
                        // tile ([warp][row][TW]; 128-byte rows) instead of whole rows.
                        tiles = __reduce_add_sync(FULLMASK, (uint32_t)__popc(wmask));
                        tiled = tiles * 2u <= (uint32_t)__popc(need) * CONSUMERS;
                    }
                    const uint32_t abytes = (uint32_t)nr * 16u;
                    // the item's first stage sent (not necessarily s == 0) carries its beta pairs
                    const uint32_t cbytes = first ? (uint32_t)IC * 8u : 0u;
                    const uint32_t cdata = tiled ? tiles * (uint32_t)(TW * 4) : (uint32_t)__popc(need) * ROW_BYTES;
                    const int y0 = ra - pd.roff;
                    int slot;
                    if (!next_slot(slot)) { ok = false; break; }
                    // The producer warp shares its SM's issue slots with 24 consumer
                    // warps, so every instruction between the slot becoming free and
                    // the tile's copy adds to the stage's latency: the long copy goes
                    // first, the small ones and the header after it.
                    if (lane == 0) {
                        mbar_expect(&S.full[slot], cdata + 2u * abytes + cbytes);
                        cstreamed += cdata;
                        if (!tiled && need == FULLMASK) {
                            tma_box(maps, TMA_BOXES - 1, S.stage[slot], col0, y0, &S.full[slot]);
                        } else {
                            // one run of consecutive needed rows at a time
                            uint32_t rem = tiled ? 0u : need;
                            while (rem) {
                                const int a = __ffs(rem) - 1;
                                const uint32_t x = rem >> a;
                                const int len = x == FULLMASK ? 32 : __ffs(~x) - 1;
                                tma_rows(maps, S.stage[slot] + a * IC, col0, y0 + a, len, &S.full[slot]);
                                rem &= a + len >= 32 ? 0u : ~((1u << (a + len)) - 1u);
                            }
                        }
                        bulk_copy(S.rowA[slot], A.rowA + ra, abytes, &S.full[slot]);
                        bulk_copy(S.rowG[slot], A.rowg + ra, abytes, &S.full[slot]);
                        if (first) bulk_copy(S.colB[slot], A.B2 + pd.bcoff + col0, IC * 8u, &S.full[slot]);
                        StageHdr& hh = S.hdr[slot];
                        hh.ra = ra;
                        hh.nr = nr;
                        hh.flags = first ? H_FIRST : 0;
                        hh.tiled = tiled ? 1 : 0;
                    }
                    if (screened && lane < CONSUMERS) S.rmaskw[slot][lane] = wmask;
                    if (lane < DESC_WORDS) reinterpret_cast<int*>(&S.hdr[slot].d)[lane] = w0;
                    __syncwarp();  // the transaction count is registered before the tiles' copies
                    if (tiled && lane < CONSUMERS) {
                        uint32_t rem = wmask;
                        float* dst = S.stage[slot] + lane * SR * TW;
                        while (rem) {
                            const int a = __ffs(rem) - 1;
                            const uint32_t x = rem >> a;
                            const int len = x == FULLMASK ? 32 : __ffs(~x) - 1;
                            tma_tile_rows(maps, dst + a * TW, col0 + lane * TW, y0 + a, len, &S.full[slot]);
                            rem &= a + len >= 32 ? 0u : ~((1u << (a + len)) - 1u);
                        }
                    }
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&S.full[slot]);
                    issued++;
                    first = false;
                }
            }
            if (!ok) break;
            i0 = i1; w0 = w1; a0 = a1; v0 = v1;
            i1 = i2; w1 = w2;
            i2r = i3r;
        }
        if (lane == 0 && A.c_streamed) atomicAdd(A.c_streamed, cstreamed);
        if (!ok) {
            if (lane == 0) atomicOr(A.err, 1);
            // wait (bounded, at the default limit) for the copies already issued into the ring
            for (long long k = (issued > NSTAGES ? issued - NSTAGES : 0); k < issued; k++)
                mbar_wait(&S.full[k % NSTAGES], (uint32_t)((k / NSTAGES) & 1), WAIT_NS);
        }
        return;
    }

    // ----------------------------------------------------------- consumers
    const int wc = warp * TW + lane;  // this lane's column within an item
    long long consumed = 0;
    Ctx x;
    x.bp = -INFINITY; x.colg = 0; x.U = 0u; x.real = false; x.prob = 0;
    x.r0 = 0;
    x.rend = 0;
    x.pslot = 0;
    Block blk;
    open_block(blk, make_int4(0, 0, 0, 0), false, x);
    for (;;) {
        const int slot = (int)(consumed % NSTAGES);
        if (!mbar_wait(&S.full[slot], (uint32_t)((consumed / NSTAGES) & 1), wlim)) {
            if (lane == 0) atomicOr(A.err, 2);
            return;
        }
        const StageHdr& hs = S.hdr[slot];
        const int flags = hs.flags;
        if (flags & H_TERM) return;
        const int r0 = hs.d.r0;
        if (flags & H_FIRST) {
            x.pslot = hs.d.part + hs.d.sub;
            x.prob = hs.d.prob;
            const ProbDesc pd = A.inline_maps ? A.pd0 : A.probs[x.prob];
            x.colg = pd.coff + hs.d.col0 + wc;
            x.real = wc < hs.d.ncols;
            // B'; no element of a missing column (past the problem's last one, where the
            // pairs may be another problem's) passes
            x.bp = x.real ? bound_up(S.colB[slot][wc].x) : -INFINITY;
            blk.gend = r0;  // no block continues into the item
        }
        x.r0 = r0;
        x.rend = r0 + hs.d.rows;
        x.ra = hs.ra;
        x.nr = hs.nr;
        const bool tiled = hs.tiled != 0;
        x.rs = tiled ? TW : IC;
        x.st = S.stage[slot] + (tiled ? warp * SR * TW + lane : wc);
        x.rA = S.rowA[slot];
        const int4* rG = S.rowG[slot];
        const uint32_t wrows = A.unit_need ? S.rmaskw[slot][warp] : FULLMASK;  // rows this warp evaluates
        if (wrows == 0u) {
            // screened, and no block of this warp's tile in the stage is needed: a
            // needed block that continued here or started here would have rows in
            // wrows, so nothing is open for this warp past the stage
            blk.gend = x.ra + x.nr;
        } else if (SNAP) {
            // every block: z~ and o~ of Def. 1 for the snapshot
            int r = 0;
            while (r < x.nr) {
                if (x.ra + r == blk.gend) open_block(blk, rG[r], (wrows >> r) & 1u, x);
                const int e = min(blk.gend - x.ra, x.nr);
                if (blk.need) scan_rows(blk, x, r, e);
                r = e;
                if (x.ra + r == blk.gend && blk.need) finish_block<true>(A, blk, x, lane);
            }
        } else {
            // only the groups with a marked chunk (and a block that ends here):
            // an unmarked chunk has y <= 0 in every row, so it adds nothing
            const uint32_t live = (x.nr >= SR ? 0xffu : (1u << ((x.nr + 3) >> 2)) - 1u) & chunks_of_rows(wrows);
            const uint32_t cm = tiled ? chunk_marks<TW>(x.st, x.rA, x.bp) : chunk_marks<IC>(x.st, x.rA, x.bp);
            x.U = __reduce_or_sync(FULLMASK, cm & live);
            int r = 0;
            bool cont = blk.gend > x.ra;  // the block open at the end of the last stage continues here
            while (cont || r < x.nr) {
                int s0 = 0;
                if (!cont) {
                    // the group of the first marked chunk at or after r (it starts at or
                    // after r); with none, the stage's last group, which stays open (with
                    // nothing summed) in case it continues -- a piece of a split group
                    // still reports (zero) partial sums at its end
                    const uint32_t Ur = x.U & ~((1u << (r >> 2)) - 1u);
                    const int rc = Ur ? max(r, 4 * (__ffs(Ur) - 1)) : x.nr - 1;
                    open_block(blk, rG[rc], (wrows >> rc) & 1u, x);
                    s0 = blk.gstart - x.ra;
                }
                cont = false;
                const int e = min(blk.gend - x.ra, x.nr);
                if (blk.need) block_marked_rows(blk, x, s0, e);
                if (blk.gend <= x.ra + x.nr && blk.need) finish_block<false>(A, blk, x, lane);
                r = e;
            }
        }
        __syncwarp();
        if (lane == 0 && !A.stall) mbar_arrive(&S.empty[slot]);
        consumed++;
    }
}

// ========================================================== stage masks
// Screened evaluations: per (item, stage, row) the needed tiles of the item
// for the row's group (bit w = tile w of the item's 256 columns), from the
// unit bitmask, so that the evaluation kernel's producer reads them without
// a chain of dependent loads.  One block per active item.
static_assert(SR == 32, "k_stage_masks: a warp covers one stage");
__global__ void __launch_bounds__(256) k_stage_masks(const EvalArgs A)
{
    if (A.gate && !*A.gate) return;
    if (A.ctl->wl) return;
    for (int it = blockIdx.x; it < A.nlist; it += gridDim.x) {
        const ItemDesc d = A.desc[it];
        if (A.item_active && !A.item_active[d.item]) continue;  // (uniform)
        const int tile0 = d.col0 / TW;  // a multiple of NWARPS: the item's tiles share one mask word
        uint8_t* out = const_cast<uint8_t*>(A.stage_m8) + (int64_t)d.sbase * SR;
        // a warp's 32 entries are one stage's rows (SR == 32): the stage's bit in
        // stage_need is set when some row is needed, else cleared
        for (int q = threadIdx.x; q < d.nst * SR; q += blockDim.x) {
            const int st = q / SR, i = q % SR;
            const int ra = A.stage_row0[d.st0 + st], re = A.stage_row0[d.st0 + st + 1];
            uint32_t m8 = 0u;
            if (ra + i < re) {
                const int l = A.rowg[ra + i].x;
                m8 = (A.unit_need[(int64_t)l * A.unit_words + (tile0 >> 5)] >> (tile0 & 31)) & 0xffu;
            }
            out[q] = (uint8_t)m8;
            const bool any = __ballot_sync(FULLMASK, m8 != 0u) != 0u;
            if ((threadIdx.x & 31) == 0) {
                const int gs = d.sbase + st;
                if (any) atomicOr(A.stage_need + (gs >> 5), 1u << (gs & 31));
                else atomicAnd(A.stage_need + (gs >> 5), ~(1u << (gs & 31)));
            }
        }
    }
}

void launch_stage_masks(const EvalArgs& a, int n_sm, cudaStream_t st)
{
    // a grid of a few CTAs per SM: when the screen took the block-set route
    // the kernel returns at once, and few CTAs return sooner than thousands
    k_stage_masks<<<std::min(a.nlist, 4 * n_sm), 256, 0, st>>>(a);
}

// ========================================================== split finish
// One CTA per block set at a time, warp w = tile w of the set's 256 columns:
// add the pieces' FP32 bound sums (and the snapshot's [y]_-^2 sums) in piece
// order, then, as the evaluation kernel does for a block that ends in its
// ring: the flagged blocks go to the exact-sum kernel, and a snapshot stores
// the bound as z~ (replaced by the exact value for flagged blocks) and o~.
__global__ void __launch_bounds__(NWARPS * 32) k_split_finish(const EvalArgs A)
{
    if (A.gate && !*A.gate) return;
    if (A.ctl->wl) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int si = blockIdx.x; si < A.nsets; si += gridDim.x) {
        const SplitSet st = A.sets[si];
        if (A.prob_active && !A.prob_active[st.prob]) continue;  // a finished problem of a batch
        const ProbDesc pd = A.inline_maps ? A.pd0 : A.probs[st.prob];
        const int tile = st.col0 / TW + warp;  // within the problem
        if (A.unit_need && !((A.unit_need[(int64_t)st.l * A.unit_words + (tile >> 5)] >> (tile & 31)) & 1u))
            continue;  // a screened-out unit: its pieces wrote nothing this evaluation
        const int lcol = st.col0 + warp * TW + lane;
        const int colg = pd.coff + lcol;
        const bool real = lcol < pd.n;
        float sp = 0.f, o = 0.f;
        for (int k = 0; k < st.split; k++) {
            const float* q = A.split_part + ((int64_t)(st.part + k) * ITEM_COLS + warp * TW + lane) * SPLIT_VALS;
            sp = __fadd_rn(sp, q[0]);
            o = __fadd_rn(o, q[1]);
        }
        const int k = st.rend - st.rstart + st.split;
        const uint32_t fw = __ballot_sync(FULLMASK, real && flag_block(sp, k, A.thr_flag));
        if (fw) add_xentry(A, st.rstart, st.rend, colg - lane, st.prob, st.l, fw, lane);
        if (A.zt) put_snap(A, st.l, colg, real, sp_up(sp, k), __fsqrt_ru(o));
    }
}

// (a screened evaluation on the block-set route returns from it at once: a
// grid of hundreds of CTAs, not thousands, keeps that short)
constexpr int SPLIT_FINISH_CTAS = 608;

void launch_split_finish(const EvalArgs& a, cudaStream_t st)
{
    if (a.nsets > 0) k_split_finish<<<a.nsets < SPLIT_FINISH_CTAS ? a.nsets : SPLIT_FINISH_CTAS, NWARPS * 32, 0, st>>>(a);
}

// ============================================================ exact sums
// The flagged blocks of classes of at most XTALL_ROWS rows: one warp per
// entry (a group's rows x up to 32 columns of a tile), up to XCOLS of its
// columns per sweep, one row per lane (rows gstart + lane + 32 u).  First sweep: each lane sums S = sum [f]_+^2 and
// P = sum [f]_+ over its rows in double-float (f formed with TwoSum where the
// bound y > 0), the warp adds the lanes' sums in a fixed xor tree, and Eq. 5
// gives s and psi (psi in fixed point into the problem's accumulators, the
// column sum s P in fixed point, the snapshot's z~).  Second sweep, where
// some s > 0, over the same rows (now in L1/L2): the nonzero t_ij = s
// [f_ij]_+ of the row, summed over the sweep's columns, to the row's
// fixed-point sum (consecutive rows: one coalesced atomic per 32 rows).  C is
// read in 32-byte sectors of the active columns only; the alpha records are
// coalesced; XUNROLL rows per lane are in flight.  The block decomposition
// and the order of every floating-point sum are fixed, so results do not
// depend on scheduling.
constexpr int EXACT_THREADS = 256;
constexpr int XCOLS = 2;
static_assert(XCOLS == 2, "the tall-class kernel finishes column q on thread q");
constexpr int XUNROLL = 4;

// The warp's sum of a double-float value, in a fixed xor tree; lane 0's result.
__device__ __forceinline__ void warp_df_sum(float& h, float& l)
{
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        const float oh = __shfl_xor_sync(FULLMASK, h, off), ol = __shfl_xor_sync(FULLMASK, l, off);
        df_add(h, l, oh, ol);
    }
    h = __shfl_sync(FULLMASK, h, 0);
    l = __shfl_sync(FULLMASK, l, 0);
}

__global__ void __launch_bounds__(EXACT_THREADS, 2) k_exact(const EvalArgs A)
{
    if (A.gate && !*A.gate) return;
    const int ne = min(A.ctl->nxent, A.xent_cap);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = EXACT_THREADS / 32;
    __shared__ FxScale fx1;  // one problem: the evaluation's scale
    if (threadIdx.x == 0 && !A.pfx && ne > 0) fx1 = fx_scale(A.ctl->amax, A.ctl->bmax, A.fx_m, A.fx_n, A.gamma);
    __syncthreads();
    int pprob = -1;          // the problem of the psi sums held by lane 0
    long long ph = 0, pl = 0;
    for (int t = blockIdx.x * nw + warp; t < ne; t += gridDim.x * nw) {
        const XEntry E = A.xent[t];
        const ProbDesc pd = A.inline_maps ? A.pd0 : A.probs[E.prob];
        const FxScale& fx = A.pfx ? A.pfx[E.prob] : fx1;
        if (E.prob != pprob) {  // psi of another problem: flush the held sums
            if (lane == 0 && (ph | pl) != 0) {
                atomicAdd(A.psix + 2 * pprob, (unsigned long long)ph);
                atomicAdd(A.psix + 2 * pprob + 1, (unsigned long long)pl);
            }
            ph = pl = 0;
            pprob = E.prob;
        }
        uint32_t rem = E.mask;  // columns of the problem only
        while (rem) {
            int kc[XCOLS];
            float bh[XCOLS], bl[XCOLS], bp[XCOLS];
            const float* cp[XCOLS];
#pragma unroll
            for (int q = 0; q < XCOLS; q++) {
                kc[q] = rem ? __ffs(rem) - 1 : -1;
                rem &= rem - 1u;
                const int lcol = E.colg0 + max(kc[q], 0) - pd.coff;
                const float2 b2 = kc[q] >= 0 ? __ldg(A.B2 + pd.bcoff + lcol) : make_float2(0.f, 0.f);
                bh[q] = b2.x;
                bl[q] = b2.y;
                bp[q] = kc[q] >= 0 ? bound_up(b2.x) : -INFINITY;
                cp[q] = pd.C + lcol - (int64_t)pd.roff * pd.ldc;  // row R of the problem at cp + R ldc
            }
            Acc acc[XCOLS];
#pragma unroll
            for (int q = 0; q < XCOLS; q++) acc[q] = Acc{0.f, 0.f, 0.f, 0.f};
            for (int R0 = E.gstart; R0 < E.gend; R0 += 32 * XUNROLL) {
                float c[XUNROLL][XCOLS];
                float4 a[XUNROLL];
#pragma unroll
                for (int u = 0; u < XUNROLL; u++) {
                    const int R = R0 + 32 * u + lane;
                    const bool in = R < E.gend;
                    a[u] = in ? __ldg(A.rowA + R) : make_float4(0.f, 0.f, -INFINITY, 0.f);
#pragma unroll
                    for (int q = 0; q < XCOLS; q++) c[u][q] = (in && kc[q] >= 0) ? __ldg(cp[q] + (int64_t)R * pd.ldc) : 0.f;
                }
#pragma unroll
                for (int u = 0; u < XUNROLL; u++)
#pragma unroll
                    for (int q = 0; q < XCOLS; q++)
                        if (maybe_pos(a[u].z, c[u][q], bp[q])) {
                            float fh, fl;
                            f_exact(a[u].x, a[u].y, bh[q], bl[q], c[u][q], fh, fl);
                            if (fh > 0.f) acc_p(fh, fl, acc[q]);
                        }
            }
            float s[XCOLS];
            bool anys = false;
#pragma unroll
            for (int q = 0; q < XCOLS; q++) {
                s[q] = 0.f;
                if (kc[q] < 0) continue;  // (uniform)
                warp_df_sum(acc[q].Sh, acc[q].Sl);
                warp_df_sum(acc[q].Ph, acc[q].Pl);
                float psh, psl;
                s[q] = block_scale(acc[q].Sh, acc[q].Sl, A, psh, psl);
                anys = anys || s[q] > 0.f;
                if (lane == 0) {
                    const int colg = E.colg0 + kc[q];
                    if (s[q] > 0.f) {
                        psi_to_fx(psh, psl, fx.to_p, ph, pl);
                        atomicAdd(A.colfx + colg, (unsigned long long)col_q(s[q], acc[q].Ph, acc[q].Pl, fx.to_cf));
                    }
                    if (A.zt) A.zt[(int64_t)E.l * A.ntiles * TW + colg] = z_up(acc[q].Sh, acc[q].Sl);
                }
            }
            if (!anys) continue;  // (uniform)
            for (int R0 = E.gstart; R0 < E.gend; R0 += 32 * XUNROLL) {
                float c[XUNROLL][XCOLS];
                float4 a[XUNROLL];
#pragma unroll
                for (int u = 0; u < XUNROLL; u++) {
                    const int R = R0 + 32 * u + lane;
                    const bool in = R < E.gend;
                    a[u] = in ? __ldg(A.rowA + R) : make_float4(0.f, 0.f, -INFINITY, 0.f);
#pragma unroll
                    for (int q = 0; q < XCOLS; q++)
                        c[u][q] = (in && s[q] > 0.f) ? __ldg(cp[q] + (int64_t)R * pd.ldc) : 0.f;
                }
#pragma unroll
                for (int u = 0; u < XUNROLL; u++) {
                    unsigned long long tq = 0ull;
#pragma unroll
                    for (int q = 0; q < XCOLS; q++)
                        if (s[q] > 0.f && maybe_pos(a[u].z, c[u][q], bp[q])) {
                            float fh, fl;
                            f_exact(a[u].x, a[u].y, bh[q], bl[q], c[u][q], fh, fl);
                            if (fh > 0.f) tq += t_q(__fmul_rn(s[q], fh), fx.to_rf);
                        }
                    if (tq) atomicAdd(A.rowfx + R0 + 32 * u + lane, tq);
                }
            }
        }
    }
    if (lane == 0 && pprob >= 0 && (ph | pl) != 0) {
        atomicAdd(A.psix + 2 * pprob, (unsigned long long)ph);
        atomicAdd(A.psix + 2 * pprob + 1, (unsigned long long)pl);
    }
}

// Classes taller than XTALL_ROWS: one CTA of TALL_THREADS per block set at a
// time, thread t taking rows gstart + t + TALL_THREADS u; all of a class's
// loads of a sweep (up to XT_CACHED_ROWS rows) are in flight together.  The
// CTA's sums: each warp's fixed xor tree, then the warps' sums in warp order
// (thread q finishes column q).  The first sweep keeps the positive parts
// [f]_+ (hi) of its first XT_CACHED_ROWS rows in shared memory, so the second
// sweep reads C again only for rows past them.
constexpr int TALL_THREADS = 256;
constexpr int XT_UNROLL = 8;
constexpr int XT_SLOTS = 16;  // rows per thread kept
constexpr int XT_CACHED_ROWS = TALL_THREADS * XT_SLOTS;

__global__ void __launch_bounds__(TALL_THREADS, 2) k_exact_tall(const EvalArgs A)
{
    if (A.gate && !*A.gate) return;
    const int ne = min(A.ctl->nxtall, A.xtall_cap);
    constexpr int NW = TALL_THREADS / 32;
    __shared__ float red[NW][XCOLS][4];
    __shared__ float sv[XCOLS];
    __shared__ float fkeep[XT_SLOTS][XCOLS][TALL_THREADS];  // [row slot][column][thread]: [f]_+ hi
    __shared__ FxScale fx1;  // one problem: the evaluation's scale
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0 && !A.pfx && ne > 0) fx1 = fx_scale(A.ctl->amax, A.ctl->bmax, A.fx_m, A.fx_n, A.gamma);
    __syncthreads();
    int pprob = -1;  // thread q < XCOLS: the problem of the psi sums it holds
    long long ph = 0, pl = 0;
    for (int t = blockIdx.x; t < ne; t += gridDim.x) {
        const XEntry E = A.xtall[t];
        const ProbDesc pd = A.inline_maps ? A.pd0 : A.probs[E.prob];
        const FxScale& fx = A.pfx ? A.pfx[E.prob] : fx1;
        if (E.prob != pprob) {
            if (tid < XCOLS && (ph | pl) != 0) {
                atomicAdd(A.psix + 2 * pprob, (unsigned long long)ph);
                atomicAdd(A.psix + 2 * pprob + 1, (unsigned long long)pl);
            }
            ph = pl = 0;
            pprob = E.prob;
        }
        uint32_t rem = E.mask;
        while (rem) {
            int kc[XCOLS];
            float bh[XCOLS], bl[XCOLS], bp[XCOLS];
            const float* cp[XCOLS];
#pragma unroll
            for (int q = 0; q < XCOLS; q++) {
                kc[q] = rem ? __ffs(rem) - 1 : -1;
                rem &= rem - 1u;
                const int lcol = E.colg0 + max(kc[q], 0) - pd.coff;
                const float2 b2 = kc[q] >= 0 ? __ldg(A.B2 + pd.bcoff + lcol) : make_float2(0.f, 0.f);
                bh[q] = b2.x;
                bl[q] = b2.y;
                bp[q] = kc[q] >= 0 ? bound_up(b2.x) : -INFINITY;
                cp[q] = pd.C + lcol - (int64_t)pd.roff * pd.ldc;
            }
            Acc acc[XCOLS];
#pragma unroll
            for (int q = 0; q < XCOLS; q++) acc[q] = Acc{0.f, 0.f, 0.f, 0.f};
            for (int R0 = E.gstart; R0 < E.gend; R0 += TALL_THREADS * XT_UNROLL) {
                float c[XT_UNROLL][XCOLS];
                float ax[XT_UNROLL], ay[XT_UNROLL], az[XT_UNROLL];
#pragma unroll
                for (int u = 0; u < XT_UNROLL; u++) {
                    const int R = R0 + TALL_THREADS * u + tid;
                    const bool in = R < E.gend;
                    const float4 a = in ? __ldg(A.rowA + R) : make_float4(0.f, 0.f, -INFINITY, 0.f);
                    ax[u] = a.x;
                    ay[u] = a.y;
                    az[u] = a.z;
#pragma unroll
                    for (int q = 0; q < XCOLS; q++) c[u][q] = (in && kc[q] >= 0) ? __ldg(cp[q] + (int64_t)R * pd.ldc) : 0.f;
                }
                const int slot0 = (R0 - E.gstart) / TALL_THREADS;  // the same for the whole CTA
#pragma unroll
                for (int u = 0; u < XT_UNROLL; u++) {
#pragma unroll
                    for (int q = 0; q < XCOLS; q++) {
                        float fk = 0.f;
                        if (maybe_pos(az[u], c[u][q], bp[q])) {
                            float fh, fl;
                            f_exact(ax[u], ay[u], bh[q], bl[q], c[u][q], fh, fl);
                            if (fh > 0.f) {
                                acc_p(fh, fl, acc[q]);
                                fk = fh;
                            }
                        }
                        if (slot0 + u < XT_SLOTS) fkeep[slot0 + u][q][tid] = fk;
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < XCOLS; q++) {
                if (kc[q] < 0) continue;  // (uniform)
                warp_df_sum(acc[q].Sh, acc[q].Sl);
                warp_df_sum(acc[q].Ph, acc[q].Pl);
                if (lane == 0) {
                    red[warp][q][0] = acc[q].Sh;
                    red[warp][q][1] = acc[q].Sl;
                    red[warp][q][2] = acc[q].Ph;
                    red[warp][q][3] = acc[q].Pl;
                }
            }
            __syncthreads();
            if (tid < XCOLS) {  // thread q: column q
                const int q = tid;
                const int kq = q == 0 ? kc[0] : kc[XCOLS - 1];
                float sq = 0.f;
                if (kq >= 0) {
                    Acc T = {0.f, 0.f, 0.f, 0.f};
                    for (int w = 0; w < NW; w++) {  // in warp order
                        df_add(T.Sh, T.Sl, red[w][q][0], red[w][q][1]);
                        df_add(T.Ph, T.Pl, red[w][q][2], red[w][q][3]);
                    }
                    float psh, psl;
                    sq = block_scale(T.Sh, T.Sl, A, psh, psl);
                    const int colg = E.colg0 + kq;
                    if (sq > 0.f) {
                        psi_to_fx(psh, psl, fx.to_p, ph, pl);
                        atomicAdd(A.colfx + colg, (unsigned long long)col_q(sq, T.Ph, T.Pl, fx.to_cf));
                    }
                    if (A.zt) A.zt[(int64_t)E.l * A.ntiles * TW + colg] = z_up(T.Sh, T.Sl);
                }
                sv[q] = sq;
            }
            __syncthreads();
            float s[XCOLS];
            bool anys = false;
#pragma unroll
            for (int q = 0; q < XCOLS; q++) {
                s[q] = sv[q];
                anys = anys || s[q] > 0.f;
            }
            if (anys) {  // (uniform)
                // the kept rows: [f]_+ from shared memory
                const int kept = min(E.gend - E.gstart, XT_CACHED_ROWS);
                for (int k = 0; k < XT_SLOTS && k * TALL_THREADS < kept; k++) {
                    const int R = E.gstart + TALL_THREADS * k + tid;
                    unsigned long long tq = 0ull;
#pragma unroll
                    for (int q = 0; q < XCOLS; q++) {
                        const float fh = fkeep[k][q][tid];
                        if (s[q] > 0.f && fh > 0.f) tq += t_q(__fmul_rn(s[q], fh), fx.to_rf);
                    }
                    if (tq) atomicAdd(A.rowfx + R, tq);  // (fh > 0 only for rows of the set)
                }
                // the rows past them: C again
                for (int R0 = E.gstart + XT_CACHED_ROWS; R0 < E.gend; R0 += TALL_THREADS * XT_UNROLL) {
#pragma unroll
                    for (int u = 0; u < XT_UNROLL; u++) {
                        const int R = R0 + TALL_THREADS * u + tid;
                        if (R >= E.gend) break;
                        const float4 a = __ldg(A.rowA + R);
                        unsigned long long tq = 0ull;
#pragma unroll
                        for (int q = 0; q < XCOLS; q++) {
                            if (!(s[q] > 0.f)) continue;
                            const float cq = __ldg(cp[q] + (int64_t)R * pd.ldc);
                            if (maybe_pos(a.z, cq, bp[q])) {
                                float fh, fl;
                                f_exact(a.x, a.y, bh[q], bl[q], cq, fh, fl);
                                if (fh > 0.f) tq += t_q(__fmul_rn(s[q], fh), fx.to_rf);
                            }
                        }
                        if (tq) atomicAdd(A.rowfx + R, tq);
                    }
                }
            }
            __syncthreads();  // red, sv and fkeep are reused by the next columns
        }
    }
    if (tid < XCOLS && pprob >= 0 && (ph | pl) != 0) {
        atomicAdd(A.psix + 2 * pprob, (unsigned long long)ph);
        atomicAdd(A.psix + 2 * pprob + 1, (unsigned long long)pl);
    }
}

// The flagged block sets read from the transposed copy of C, where block
// (l, j) is the contiguous run CT[j][gstart, gend) of its problem: warps read
// it with coalesced loads, one row per lane, and only the flagged columns'
// bytes are read.
//  * A taller class's column (a column task): one warp, taken from a counter
//    before the shorter sets (the longest work goes out first).  Lane k takes
//    rows gstart + k, gstart + k + 32, ... in that order, XSLICE rows a load
//    round, and sums S = sum [f]_+^2 and P = sum [f]_+ in double-float; the
//    lanes' sums are then added in the fixed xor tree, and the block is
//    finished (Eq. 5: psi in fixed point, the column sum s P, a snapshot's
//    z~).  Each lane also keeps its rows' [f]_+ (the float pair's high part,
//    which is all t_ij = s [f_ij]_+ uses) in the warp's XT_CACHE floats of
//    shared memory, so the rows' t_ij go to the row sums without a second
//    read of C; rows past the cache are formed again from C.
//  * A shorter class's set (at most XTALL_ROWS rows): one warp, taken from a
//    counter.  Per column the same sums over its rows (one slice), Eq. 5, the
//    first XS_CACHED columns' [f]_+ kept in the warp's cache; then per row the
//    t_ij of every column with s > 0 (kept ones from the cache, the others
//    formed again from C), one atomic per row.
// Every floating-point sum has a fixed order, so a block's results do not
// depend on its set, on scheduling or on the evaluation being screened.
constexpr int XTC_THREADS = 256;
constexpr int XTC_UNROLL = 8;
constexpr int XT_CACHE = 2048;  // rows of a taller class's column whose [f]_+ a warp keeps (8 KB)
static_assert(XSLICE == 32 * XTC_UNROLL, "a slice is one load round of a warp");
static_assert(XT_CACHE % XSLICE == 0, "the cache ends at a slice boundary");
constexpr size_t exact_t_smem_bytes() { return sizeof(float) * XT_CACHE * (XTC_THREADS / 32); }
constexpr int XS_CACHED = XT_CACHE / XSLICE;  // columns of a shorter class's set whose [f]_+ a warp keeps
static_assert(XTALL_ROWS <= XSLICE, "a shorter class's column fits one cache slot");

// Eq. 5 for one block from its sums (lane 0's work): psi into (ph, pl), s P
// into the column sum, a snapshot's z~.  Returns s.
__device__ __forceinline__ float finish_block_exact(const EvalArgs& A, const FxScale& fx, const Acc& T, int l,
                                                    int colg, long long& ph, long long& pl)
{
    float psh, psl;
    const float s = block_scale(T.Sh, T.Sl, A, psh, psl);
    if (s > 0.f) {
        psi_to_fx(psh, psl, fx.to_p, ph, pl);
        atomicAdd(A.colfx + colg, (unsigned long long)col_q(s, T.Ph, T.Pl, fx.to_cf));
    }
    if (A.zt) A.zt[(int64_t)l * A.ntiles * TW + colg] = z_up(T.Sh, T.Sl);
    return s;
}

__device__ __forceinline__ void hold_psi(const EvalArgs& A, int prob, int& pprob, long long& ph, long long& pl)
{
    if (prob != pprob) {
        if (pprob >= 0 && (ph | pl) != 0) {
            atomicAdd(A.psix + 2 * pprob, (unsigned long long)ph);
            atomicAdd(A.psix + 2 * pprob + 1, (unsigned long long)pl);
        }
        ph = pl = 0;
        pprob = prob;
    }
}

// One load round of a column of CT: rows a0 + 32 u + lane (below r1) of the
// column and their (alpha hi, lo); A' = bound_up(alpha hi) is formed where
// it is used (it is the row record's third field, bit for bit).
__device__ __forceinline__ void load_rows(const EvalArgs& A, const float* col, int a0, int r1, int lane,
                                          float2 (&a)[XTC_UNROLL], float (&c)[XTC_UNROLL])
{
#pragma unroll
    for (int u = 0; u < XTC_UNROLL; u++) {
        const int R = a0 + 32 * u + lane;
        const bool in = R < r1;
        a[u] = in ? __ldg(reinterpret_cast<const float2*>(A.rowA + R)) : make_float2(0.f, 0.f);
        c[u] = in ? __ldg(col + R) : 0.f;
    }
}

__global__ void __launch_bounds__(XTC_THREADS, 3) k_exact_t(const EvalArgs A)
{
    if (A.gate && !*A.gate) return;
    const int nx = min(A.ctl->nxent, A.xent_cap);
    const int ntc = min(A.ctl->ntcol, A.xtcol_cap);
    const int tid = threadIdx.x, lane = tid & 31;
    __shared__ FxScale fx1;  // one problem: the evaluation's scale
    extern __shared__ float xcache[];                // XT_CACHE floats per warp
    float* fk = xcache + (tid >> 5) * XT_CACHE;      // this warp's: [f]_+ of a column's rows, by row
    if (tid == 0 && !A.pfx && nx + ntc > 0) fx1 = fx_scale(A.ctl->amax, A.ctl->bmax, A.fx_m, A.fx_n, A.gamma);
    __syncthreads();
    int pprob = -1;  // lane 0 of each warp: the problem of the psi sums it holds
    long long ph = 0, pl = 0;
    // the taller classes' columns, a warp each
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(&A.ctl->tnext, 1);
        t = __shfl_sync(FULLMASK, t, 0);
        if (t >= ntc) break;
        const XEntry E = A.xtall[A.xtmap[t]];
        const ProbDesc& pd = A.inline_maps ? A.pd0 : A.probs[E.prob];
        const FxScale& fx = A.pfx ? A.pfx[E.prob] : fx1;
        const int k = __fns(E.mask, 0, t - E.tbase + 1);  // the column of this task
        const int lcol = E.colg0 + k - pd.coff;
        const float2 b2 = __ldg(A.B2 + pd.bcoff + lcol);
        const float bp = bound_up(b2.x);
        const float* col = pd.CT + (int64_t)lcol * pd.ldct - pd.roff;
        Acc T = {0.f, 0.f, 0.f, 0.f};  // this lane's rows, in row order
        // each round's loads go out before the previous round is summed
        float2 an[XTC_UNROLL];
        float cn[XTC_UNROLL];
        load_rows(A, col, E.gstart, E.gend, lane, an, cn);
        for (int a0 = E.gstart; a0 < E.gend; a0 += XSLICE) {
            float2 a[XTC_UNROLL];
            float c[XTC_UNROLL];
#pragma unroll
            for (int u = 0; u < XTC_UNROLL; u++) {
                a[u] = an[u];
                c[u] = cn[u];
            }
            if (a0 + XSLICE < E.gend) load_rows(A, col, a0 + XSLICE, E.gend, lane, an, cn);
            const bool keep = a0 - E.gstart < XT_CACHE;  // (uniform)
#pragma unroll
            for (int u = 0; u < XTC_UNROLL; u++) {
                float fp = 0.f;
                if (a0 + 32 * u + lane < E.gend && maybe_pos(bound_up(a[u].x), c[u], bp)) {
                    float fh, fl;
                    f_exact(a[u].x, a[u].y, b2.x, b2.y, c[u], fh, fl);
                    if (fh > 0.f) {
                        acc_p(fh, fl, T);
                        fp = fh;
                    }
                }
                if (keep) fk[a0 - E.gstart + 32 * u + lane] = fp;
            }
        }
        warp_df_sum(T.Sh, T.Sl);
        warp_df_sum(T.Ph, T.Pl);
        float s = 0.f;
        if (lane == 0) {
            hold_psi(A, E.prob, pprob, ph, pl);
            s = finish_block_exact(A, fx, T, E.l, E.colg0 + k, ph, pl);
        }
        s = __shfl_sync(FULLMASK, s, 0);
        if (!(s > 0.f)) continue;  // (uniform)
        // t_ij = s [f_ij]_+ into the row sums: each lane reads back the rows it kept
        const int kept = min(E.gend, E.gstart + XT_CACHE);
        for (int a0 = E.gstart; a0 < kept; a0 += XSLICE) {
#pragma unroll
            for (int u = 0; u < XTC_UNROLL; u++) {
                const int R = a0 + 32 * u + lane;
                const float fh = fk[R - E.gstart];
                if (R < E.gend && fh > 0.f) atomicAdd(A.rowfx + R, t_q(__fmul_rn(s, fh), fx.to_rf));
            }
        }
        for (int a0 = kept; a0 < E.gend; a0 += XSLICE) {
            float2 a[XTC_UNROLL];
            float c[XTC_UNROLL];
            load_rows(A, col, a0, E.gend, lane, a, c);
#pragma unroll
            for (int u = 0; u < XTC_UNROLL; u++)
                if (a0 + 32 * u + lane < E.gend && maybe_pos(bound_up(a[u].x), c[u], bp)) {
                    float fh, fl;
                    f_exact(a[u].x, a[u].y, b2.x, b2.y, c[u], fh, fl);
                    if (fh > 0.f) atomicAdd(A.rowfx + a0 + 32 * u + lane, t_q(__fmul_rn(s, fh), fx.to_rf));
                }
        }
    }
    // the shorter classes' sets, a warp each
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(&A.ctl->xnext, 1);
        t = __shfl_sync(FULLMASK, t, 0);
        if (t >= nx) break;
        const XEntry E = A.xent[t];
        const ProbDesc& pd = A.inline_maps ? A.pd0 : A.probs[E.prob];
        const FxScale& fx = A.pfx ? A.pfx[E.prob] : fx1;
        if (lane == 0) hold_psi(A, E.prob, pprob, ph, pl);
        const float* ct0 = pd.CT + (int64_t)(E.colg0 - pd.coff) * pd.ldct - pd.roff;  // + k ldct + R
        // the set's rows (at most XTALL_ROWS = 32 XTC_UNROLL): their records once, and
        // each column's values loaded one column ahead of its sums
        float2 a[XTC_UNROLL];
        float ap[XTC_UNROLL];  // A' of the rows (-inf past the set)
#pragma unroll
        for (int u = 0; u < XTC_UNROLL; u++) {
            const int R = E.gstart + 32 * u + lane;
            a[u] = R < E.gend ? __ldg(reinterpret_cast<const float2*>(A.rowA + R)) : make_float2(0.f, 0.f);
            ap[u] = R < E.gend ? bound_up(a[u].x) : -INFINITY;
        }
        auto load_col = [&](int k, float (&c)[XTC_UNROLL]) {
            const float* col = ct0 + (int64_t)k * pd.ldct;
#pragma unroll
            for (int u = 0; u < XTC_UNROLL; u++) {
                const int R = E.gstart + 32 * u + lane;
                c[u] = R < E.gend ? __ldg(col + R) : 0.f;
            }
        };
        float sk = 0.f;         // lane k: s of column k
        int sq = XS_CACHED;     // lane k: column k's slot in the warp's cache (XS_CACHED: none)
        int q = 0;              // columns summed so far
        uint32_t rem = E.mask;
        float cn[XTC_UNROLL];
        if (rem) load_col(__ffs(rem) - 1, cn);
        while (rem) {
            const int k = __ffs(rem) - 1;
            rem &= rem - 1u;
            const bool keep = q < XS_CACHED;  // (uniform)
            float c[XTC_UNROLL];
#pragma unroll
            for (int u = 0; u < XTC_UNROLL; u++) c[u] = cn[u];
            if (rem) load_col(__ffs(rem) - 1, cn);
            const float2 b2 = __ldg(A.B2 + pd.bcoff + E.colg0 + k - pd.coff);
            const float bp = bound_up(b2.x);
            Acc T = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int u = 0; u < XTC_UNROLL; u++) {
                float fp = 0.f;
                if (maybe_pos(ap[u], c[u], bp)) {
                    float fh, fl;
                    f_exact(a[u].x, a[u].y, b2.x, b2.y, c[u], fh, fl);
                    if (fh > 0.f) {
                        acc_p(fh, fl, T);
                        fp = fh;
                    }
                }
                if (keep) fk[q * XSLICE + 32 * u + lane] = fp;
            }
            warp_df_sum(T.Sh, T.Sl);
            warp_df_sum(T.Ph, T.Pl);
            float s = 0.f;
            if (lane == 0) s = finish_block_exact(A, fx, T, E.l, E.colg0 + k, ph, pl);
            s = __shfl_sync(FULLMASK, s, 0);
            if (lane == k) {
                sk = s;
                if (keep) sq = q;
            }
            q++;
        }
        uint32_t srem = __ballot_sync(FULLMASK, sk > 0.f);
        if (!srem) continue;  // (uniform)
        unsigned long long tq[XTC_UNROLL];
#pragma unroll
        for (int u = 0; u < XTC_UNROLL; u++) tq[u] = 0ull;
        // the columns whose [f]_+ the lanes kept: t_ij from the cache
        uint32_t crem = srem & __ballot_sync(FULLMASK, sq < XS_CACHED);
        srem &= ~crem;
        while (crem) {
            const int k = __ffs(crem) - 1;
            crem &= crem - 1u;
            const float s = __shfl_sync(FULLMASK, sk, k);
            const int qk = __shfl_sync(FULLMASK, sq, k);
#pragma unroll
            for (int u = 0; u < XTC_UNROLL; u++) {
                const float fh = fk[qk * XSLICE + 32 * u + lane];
                if (fh > 0.f) tq[u] += t_q(__fmul_rn(s, fh), fx.to_rf);
            }
        }
        // the others from C again
        if (srem) load_col(__ffs(srem) - 1, cn);
        while (srem) {
            const int k = __ffs(srem) - 1;
            srem &= srem - 1u;
            float c[XTC_UNROLL];
#pragma unroll
            for (int u = 0; u < XTC_UNROLL; u++) c[u] = cn[u];
            if (srem) load_col(__ffs(srem) - 1, cn);
            const float s = __shfl_sync(FULLMASK, sk, k);
            const float2 b2 = __ldg(A.B2 + pd.bcoff + E.colg0 + k - pd.coff);
            const float bp = bound_up(b2.x);
#pragma unroll
            for (int u = 0; u < XTC_UNROLL; u++)
                if (maybe_pos(ap[u], c[u], bp)) {
                    float fh, fl;
                    f_exact(a[u].x, a[u].y, b2.x, b2.y, c[u], fh, fl);
                    if (fh > 0.f) tq[u] += t_q(__fmul_rn(s, fh), fx.to_rf);
                }
        }
#pragma unroll
        for (int u = 0; u < XTC_UNROLL; u++)
            if (tq[u]) atomicAdd(A.rowfx + E.gstart + 32 * u + lane, tq[u]);
    }
    if (lane == 0 && pprob >= 0 && (ph | pl) != 0) {
        atomicAdd(A.psix + 2 * pprob, (unsigned long long)ph);
        atomicAdd(A.psix + 2 * pprob + 1, (unsigned long long)pl);
    }
}

void launch_exact(const EvalArgs& a, int n_sm, cudaStream_t st)
{
    if (a.use_ct) {
        k_exact_t<<<3 * n_sm, XTC_THREADS, exact_t_smem_bytes(), st>>>(a);
        return;
    }
    k_exact<<<4 * n_sm, EXACT_THREADS, 0, st>>>(a);
    k_exact_tall<<<2 * n_sm, TALL_THREADS, 0, st>>>(a);
}

void exact_caps(const HostPlan& hp, int64_t& xent, int64_t& xtall, int64_t& tcols)
{
    xent = xtall = tcols = 0;
    for (int64_t l = 0; l < hp.L; l++) {
        const int64_t g = hp.goff[l + 1] - hp.goff[l];
        if (g == 0) continue;
        const int64_t n = hp.pn[hp.gprob[l]];
        (g > XTALL_ROWS ? xtall : xent) += (n + TW - 1) / TW;
        if (g > XTALL_ROWS) tcols += n;
    }
}

size_t stream_smem_bytes() { return sizeof(Smem) + 1024; }

bool stream_prepare()
{
    const int sm = (int)stream_smem_bytes();
    return cudaFuncSetAttribute(k_stream<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) == cudaSuccess &&
           cudaFuncSetAttribute(k_stream<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) == cudaSuccess &&
           cudaFuncSetAttribute(k_exact_t, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)exact_t_smem_bytes()) == cudaSuccess;
}

void launch_stream(const EvalArgs& a, int n_ctas, cudaStream_t st)
{
    const int sm = (int)stream_smem_bytes();
    if (a.zt) k_stream<true><<<n_ctas, THREADS, sm, st>>>(a);
    else k_stream<false><<<n_ctas, THREADS, sm, st>>>(a);
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
        for (int t = 0; t < 2; t++) {
            const cuuint32_t box[2] = {(cuuint32_t)(t ? TW : IC), 1u << k};
            CUresult r = enc(t ? &T.tile[k] : &T.box[k], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(C),
                             dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                             t ? CU_TENSOR_MAP_L2_PROMOTION_L2_128B : CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) return "cuTensorMapEncodeTiled failed with code " + std::to_string((int)r);
        }
    }
    return "";
}

}  // namespace otgs
