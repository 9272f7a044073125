// otgs_internal.cuh -- shared declarations of the CUDA path (not part of the ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstddef>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "otgs.h"

namespace otgs {

// ---------------------------------------------------------------- geometry
// A "unit" is (group l, tile of TW consecutive target columns): the
// granularity of the screening decisions (Sec. 3) and of their bitmasks.
constexpr int TW = 32;
// The evaluation kernel has NWARPS consumer warps; warp w owns tile w of an
// item's ITEM_COLS columns (one column per lane) and walks every row.
constexpr int NWARPS = 8;
constexpr int ITEM_COLS = NWARPS * TW;  // columns of a work item: 1 KB of each row of C
// C streams through a ring of NSTAGES shared-memory stages of STAGE_ROWS rows
// x ITEM_COLS columns (32 KB) per CTA, loaded by 2D TMA boxes.
constexpr int STAGE_ROWS = 32;
constexpr int NSTAGES = 2;

// CTAs of the evaluation kernel per SM (each with its own ring).  The
// consumers' per-stage work, not the bytes in flight, sets the kernel's
// speed: three CTAs of two stages (24 consumer warps, 72 registers each)
// beat two of three (16 warps, 96 registers) by 6 %, one of six by 40 %.
constexpr int CTAS_PER_SM = 3;
// Consecutive groups are packed into "panels" of whole groups up to a panel
// height; a larger group is a panel of its own.  A work item is (panel,
// column chunk of ITEM_COLS).  The height is the number of (row, column
// chunk) pairs -- m * ceil(n / ITEM_COLS) for one problem, the sum of that
// over the problems of a batch -- divided by TARGET_ITEMS and clamped to
// [MIN_PANEL_ROWS, MAX_PANEL_ROWS]: small problems get enough items to fill
// every SM; large ones stop at 128 rows (128 KB of C per item), short enough
// that the CTAs taking the last items finish close together.  On GB300 the
// evaluation kernel ran 5 % (m = n = 20000), 7 % (m = n = 10000) and 2 % (a
// batch of 512 problems) faster with 128-row panels than with 512-row ones.
constexpr int MAX_PANEL_ROWS = 128;
constexpr int MIN_PANEL_ROWS = 32;
constexpr int64_t TARGET_ITEMS = 2048;
inline int64_t row_chunks(int64_t m, int64_t n) { return m * ((n + ITEM_COLS - 1) / ITEM_COLS); }
inline int32_t panel_rows_for(int64_t row_chunk_pairs)
{
    const int64_t h = (row_chunk_pairs + TARGET_ITEMS - 1) / TARGET_ITEMS;
    return (int32_t)(h < MIN_PANEL_ROWS ? MIN_PANEL_ROWS : (h > MAX_PANEL_ROWS ? MAX_PANEL_ROWS : h));
}
inline int32_t panel_rows(int64_t m, int64_t n) { return panel_rows_for(row_chunks(m, n)); }

// Columns of the per-column float-pair split of beta, padded to whole items.
inline int32_t padded_cols(int64_t n) { return (int32_t)((n + ITEM_COLS - 1) / ITEM_COLS * ITEM_COLS); }

// alpha_i (resp. beta_j) rounded up by a relative 2^-20: with A' and B' so
// rounded, y_ij = fl(fl(A'_i - c_ij) + B'_j) >= f_ij = alpha_i + beta_j - c_ij
// whenever f_ij > 0 (then c_ij < |alpha| + |beta|, and the representation and
// rounding errors, below 6 2^-24 (|alpha| + |beta|), are covered by the 16
// 2^-24 (|alpha| + |beta|) the rounding up adds).  So [y]_+ >= [f]_+ for every
// element: y <= 0 rejects only elements whose f is certainly <= 0, and the
// FP32 sum of [y]_+^2 bounds ||[f_[l]]_+||^2 from above.
__device__ __forceinline__ float bound_up(float h) { return __fadd_ru(h, __fmul_ru(fabsf(h), 0x1p-20f)); }

// FP32 (hi, lo) split of an FP64 value: hi + lo = x to ~2^-48 relative.
__device__ __forceinline__ float2 split2(double x)
{
    const float h = __double2float_rn(x);
    return make_float2(h, __double2float_rn(x - (double)h));
}

struct EvalCtl;
// Preparation of one sorted row: (alpha hi, alpha lo, bound_up(alpha hi), 0).
// Returns [alpha hi]_+ for the fixed-point scale.
__device__ __forceinline__ float prep_row(double a, float4* rowA)
{
    const float2 s = split2(a);
    *rowA = make_float4(s.x, s.y, bound_up(s.x), 0.f);
    return fmaxf(s.x, 0.f);
}

// Preparation of one (padded) column: (beta hi, lo); a padding column gets
// (-1e30, 0).  Returns [beta hi]_+ for the fixed-point scale.
__device__ __forceinline__ float prep_col(bool real, double b, float2* B2)
{
    if (!real) {
        *B2 = make_float2(-1e30f, 0.f);
        return 0.f;
    }
    const float2 s = split2(b);
    *B2 = s;
    return fmaxf(s.x, 0.f);
}

// Groups taller than SPLIT_ROWS rows are cut into panels of SPLIT_ROWS rows
// ("pieces"), so that one block is summed by several CTAs in parallel; a
// second kernel adds the pieces' partial sums in piece order and finishes
// those blocks.
constexpr int SPLIT_ROWS = 256;

// A block set: the blocks of one split group against one 256-column chunk.
struct SplitSet {
    int l;       // group
    int col0;    // first column
    int split;   // pieces
    int part;    // partial-sum slot of piece 0 (piece k: part + k)
    int item0;   // item id of piece 0 (holds the set's psi partials)
    int rstart;  // rows of the group
    int rend;
    int prob;    // problem of a batch
};

// Values a piece of a split group stores per column: the FP32 bound sum S'
// of [y]_+^2 and the snapshot's sum of [y]_-^2.
constexpr int SPLIT_VALS = 2;

// Tunable plan parameters (0: the default rule).
struct PlanParams {
    int32_t panel_rows = 0;  // panel height (default: panel_rows(m, n))
    int32_t split_rows = 0;  // groups taller than this are cut into pieces (default: SPLIT_ROWS)
    // > 0: a stage ends early, before a group of at most STAGE_ROWS rows that
    // would straddle its end (so that the group's blocks are bounded within
    // one stage), when it keeps at least this many rows; 0 (default): stages
    // of STAGE_ROWS rows
    int32_t stage_fill = 0;
};

// A problem of a batch as the kernels see it.
struct ProbDesc {
    const float* C;  // class-sorted rows of this problem, row stride ldc
    int64_t ldc;
    const float* CT; // NULL, or its transpose: CT[j * ldct + i] = C[i * ldc + j] (block (l, j) contiguous)
    int64_t ldct;
    int32_t m, n;    // rows, columns
    int32_t roff;    // first sorted row in the concatenation
    int32_t coff;    // first column in the concatenation
    int32_t bcoff;   // first entry in the beta pair array B2 (even: 16-byte aligned bulk copies)
};

// One problem of a batch as the per-problem kernels see it (the batched
// preparation, reduction and L-BFGS step).
struct BProb {
    int32_t roff, coff, bcoff;  // first sorted row, first column, first B2 entry
    int32_t m, n;
    int32_t voff;               // first entry of the problem's solver vectors (roff + coff)
    int32_t item0, item1;       // its work items [item0, item1)
};

// A work item as the evaluation kernel sees it, in execution order (64 B).
struct ItemDesc {
    int item;   // item id (index of its active flag)
    int p;      // panel
    int r0;     // first sorted row
    int rows;   // rows (whole groups, or one piece of a split group)
    int col0;   // first column (multiple of ITEM_COLS)
    int ncols;  // columns of C in the item (<= ITEM_COLS)
    int nst;    // stages of the item's panel (at most STAGE_ROWS rows each)
    int sbase;  // first stage of the item in execution order (index into per-stage tables)
    int split;  // pieces of the item's group (1: not split)
    int sub;    // this item's piece
    int part;   // split groups: partial-sum slot of piece 0 of this block set (piece k: part + k)
    int prob;   // problem of a batch (0 for a single problem)
    int st0;    // stage s spans sorted rows [stage_row0[st0 + s], stage_row0[st0 + s + 1])
    int pad[3];
};

// ------------------------------------------------------------------ host plan
// Built once from the labels at create.  "Sorted" row r is the r-th row in
// (label, caller index) order; groups are contiguous ranges of sorted rows.
struct HostPlan {
    int64_t m = 0, n = 0;
    int32_t L = 0, ntiles = 0;
    // a batch of independent problems: rows, columns and groups are the
    // concatenation of the problems' (one problem: the trivial batch)
    int32_t nprob = 1;
    std::vector<int32_t> proff, pcoff, ploff;  // per problem: first row, column, group
    std::vector<int32_t> pm, pn;               // per problem: rows, columns
    std::vector<int32_t> pbcoff;               // per problem: first entry of B2 (columns rounded up to 4)
    int64_t nb2 = 0;                           // entries of B2, with room for a full last column chunk
    int64_t max_m = 0, max_n = 0;              // largest problem
    std::vector<int32_t> gprob;                // group -> problem
    int32_t panel_height = 0, split_height = 0, stage_fill = 0;  // the parameters the plan was built with
    std::vector<int32_t> perm;    // sorted r -> caller row
    std::vector<int32_t> goff;    // L+1 offsets (sorted rows)
    std::vector<int32_t> rgroup;  // sorted r -> group
    std::vector<int4> rowg;       // sorted r -> {group, first row, end row of the group, problem}
    // panels: row ranges of whole groups
    std::vector<int32_t> prow0;   // first sorted row
    std::vector<int32_t> prows;   // rows
    std::vector<int32_t> pprob;   // problem
    std::vector<int32_t> pW;      // columns per work item (ITEM_COLS)
    std::vector<int32_t> pnch;    // work items (column chunks) of the panel
    std::vector<int32_t> pitem;   // first work-item id of the panel
    std::vector<int32_t> psplit;  // pieces of the panel's group (1: not a piece of a split group)
    std::vector<int32_t> psub;    // the panel's piece
    std::vector<int32_t> pslot;   // pieces of split groups before the panel's group (split panels)
    std::vector<int32_t> gpanel;  // group -> panel (-1 for empty groups; the first piece if split)
    // stages: a panel's rows in runs of at most STAGE_ROWS, ended early (at
    // a group's start) rather than cut a short group in two
    std::vector<int32_t> pst0;        // panel -> its first entry of stage_row0
    std::vector<int32_t> pnst;        // panel -> its number of stages
    std::vector<int32_t> stage_row0;  // per panel: the stages' first rows, then the panel's end
    // work items, id = pitem[p] + chunk
    std::vector<int32_t> item_panel, item_chunk;
    std::vector<int32_t> exec_order;  // item ids, largest first
    std::vector<ItemDesc> desc;       // work items in execution order
    int64_t nstages = 0;              // stages streamed by one dense evaluation
    int64_t nsplit_slots = 0;         // partial-sum slots of split groups: their pieces x column chunks
    std::vector<SplitSet> sets;       // block sets of split groups
    int32_t max_group = 0;            // rows of the largest group
    bool sorted_identity = true;      // labels already non-decreasing
    int npanels() const { return (int)prows.size(); }
    int nitems() const { return (int)item_panel.size(); }
};

// Returns an empty string on success, else an error message.
std::string build_plan(const int32_t* labels, int64_t m, int64_t n, int32_t L, HostPlan& hp);
// nprob problems (host label arrays of m[k] entries in [0, L[k]), n[k] columns).
std::string build_plan_batch(int32_t nprob, const int32_t* const* labels, const int64_t* m, const int64_t* n,
                             const int32_t* L, const PlanParams& pp, HostPlan& hp);

// ---------------------------------------------------------------- device plan
struct DevPlan {
    int32_t *perm, *goff, *rgroup;
    int4* rowg;
    SplitSet* sets;
    int32_t *prows, *pW, *pnch, *pitem, *psplit, *gpanel;
    int32_t *item_panel, *item_chunk, *exec_order;
    ItemDesc* desc;
    int32_t* stage_row0;
};

// ------------------------------------------------- per-evaluation control word
// Zeroed before each evaluation's preparation kernel.
struct EvalCtl {
    int work;           // work-item counter of the evaluation kernel
    unsigned amax;      // float bits of max_i [alpha_i hi]_+
    unsigned bmax;      // float bits of max_j [beta_j hi]_+
    int nxent;          // flagged block sets of classes of at most XTALL_ROWS rows
    int nxtall;         // flagged block sets of taller classes
    int xnext;          // the next flagged block set of shorter classes for the exact-sum kernel
    int tnext;          // the next column task of the taller classes' sets
    int ntcol;          // column tasks handed out
    int wl;             // screened: 1 = the screen built the sets itself (no bound pass; see pick_route)
    unsigned long long psi[2];  // one problem: psi summed by the exact-sum kernel (fixed point, hi and lo)
    unsigned long long wl_work;  // screened: rows x columns of the blocks the screen left (see pick_route)
    unsigned long long wl_cols;  //   and their number
    unsigned wl_done;            //   CTAs of the screen kernel done (its last one picks the route)
};

// Device address of the control word's psi accumulators (host side: plain
// address arithmetic on the device pointer).
inline unsigned long long* ctl_psi(EvalCtl* c)
{
    return reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(c) + offsetof(EvalCtl, psi));
}

// Clears a control word (every field starts each evaluation at zero).
__device__ __forceinline__ void ctl_clear(EvalCtl* c)
{
    c->work = 0;
    c->amax = 0u;
    c->bmax = 0u;
    c->nxent = 0;
    c->nxtall = 0;
    c->xnext = 0;
    c->tnext = 0;
    c->ntcol = 0;
    c->wl = 0;
    c->wl_work = 0ull;
    c->wl_cols = 0ull;
    c->wl_done = 0u;
    c->psi[0] = 0ull;
    c->psi[1] = 0ull;
}

// A flagged block set for the exact-sum kernel: the blocks (group l, column
// j) of one 32-column tile whose FP32 bound does not rule out z > theta.  The
// kernel re-reads the rows [gstart, gend) for the columns in mask, forms S =
// ||[f]_+||^2 and P = sum [f]_+ in double-float, and finishes the blocks
// (Eq. 5) with their row sums.
// A flagged block set of a class taller than this goes to the exact-sum
// kernel's CTA-wide path (a warp per set for the others).
constexpr int XTALL_ROWS = 256;

struct XEntry {
    int gstart, gend;  // rows of the group
    int colg0;         // first column (in the concatenation) of the tile
    int prob;          // problem of a batch
    int l;             // group
    uint32_t mask;     // columns (bit k: column colg0 + k) to evaluate
    int tbase;         // taller classes, transposed copy: the set's first column task
    int pad_;
};

// A screened evaluation reads the blocks the screen left straight from the
// transposed copy (no bound pass) when their rows x columns are at most this
// fraction of m n.
constexpr double WL_FRACTION = 0.25;

// Rows of one load round of a warp over a column of the transposed copy
// (eight rows a lane) in the exact-sum kernel.
constexpr int XSLICE = 256;



// Adds this warp's maxima of [alpha hi]_+ and [beta hi]_+ into ctl (all
// lanes of the warp must call it).  Non-negative floats order as their bits.
__device__ __forceinline__ void record_max(EvalCtl* ctl, float apos, float bpos)
{
    const unsigned ma = __reduce_max_sync(0xffffffffu, __float_as_uint(apos));
    const unsigned mb = __reduce_max_sync(0xffffffffu, __float_as_uint(bpos));
    if ((threadIdx.x & 31) == 0) {
        if (ma) atomicMax(&ctl->amax, ma);
        if (mb) atomicMax(&ctl->bmax, mb);
    }
}

// Row and column sums of T (Eq. 5) are accumulated as int64 multiples of 2^-k,
// so their value does not depend on the order of the additions.  k comes from
// a bound on the sums: t_ij = s f_ij with s <= 1 / gamma and f_ij <= [alpha_i]_+
// + [beta_j]_+ (c >= 0), so a row sum is at most n F / gamma and a column sum
// m F / gamma, F = max [alpha]_+ + max [beta]_+; k puts that bound below 2^61.
struct FxScale {
    double to_r, from_r;  // row sums: value * to_r -> integer, integer * from_r -> value
    double to_c, from_c;  // column sums
    double to_p, from_p;  // psi: the coarse grid (its remainders go to a grid 2^30 times finer)
    float to_rf, to_cf;   // to_r, to_c as floats (exact: powers of two in FP32 range)
};

// k is kept in [-100, 100] so that 2^k is an FP32 number: a bound below
// 2^-41 only gets a coarser grid than it could, and no finite FP32 input
// gives a bound above 2^160.
__host__ __device__ inline int fx_exponent(double bound)
{
    if (!(bound > 0.0) || !(bound < 1e300)) return 0;
    const int e = ilogb(bound) + 2;  // bound < 2^(e-1): a factor 2 of slack for the FP32 split of alpha, beta
    const int k = 61 - e;
    return k < -100 ? -100 : (k > 100 ? 100 : k);
}

__host__ __device__ inline FxScale fx_scale(unsigned amax_bits, unsigned bmax_bits, int64_t m, int64_t n,
                                            float gamma)
{
    float am, bm;
#ifdef __CUDA_ARCH__
    am = __uint_as_float(amax_bits);
    bm = __uint_as_float(bmax_bits);
#else
    memcpy(&am, &amax_bits, 4);
    memcpy(&bm, &bmax_bits, 4);
#endif
    const double F = ((double)am + (double)bm) / (double)gamma;
    const int kr = fx_exponent(F * (double)n), kc = fx_exponent(F * (double)m);
    // sum psi <= sum_ij [f_ij]_+^2 / (2 gamma) <= m n F'^2 / (2 gamma), F' = (max [alpha]_+ + max [beta]_+)
    // with the 2^-20 of the bounds' rounding (a 1.01 factor of slack)
    const double Fp = ((double)am + (double)bm) * 1.01;
    const int kp = fx_exponent(Fp * Fp * (double)m * (double)n / (2.0 * (double)gamma));
    FxScale s;
    s.to_p = ldexp(1.0, kp);
    s.from_p = ldexp(1.0, -kp);
    s.to_r = ldexp(1.0, kr);
    s.from_r = ldexp(1.0, -kr);
    s.to_c = ldexp(1.0, kc);
    s.from_c = ldexp(1.0, -kc);
    s.to_rf = ldexpf(1.0f, kr);
    s.to_cf = ldexpf(1.0f, kc);
    return s;
}

// psi of one block (as the float pair of Eq. 5's evaluation) to the
// two-level fixed point of the scale: the value on the coarse grid and its
// remainder on a grid 2^30 times finer.  Each part is an exact integer
// function of the block, so sums of them do not depend on the order of the
// additions (or on which kernel formed the block).
__device__ __forceinline__ void psi_to_fx(float psh, float psl, double to_p, long long& hi, long long& lo)
{
    const double x = ((double)psh + (double)psl) * to_p;  // exact: a pair of floats, times a power of two
    const double q = rint(x);
    hi += (long long)q;
    lo += __double2ll_rn((x - q) * 1073741824.0);         // x - q is exact; |.| <= 1/2
}

// D's psi term from the fixed-point sums.
__host__ __device__ inline double psi_from_fx(long long hi, long long lo, double from_p)
{
    return (double)hi * from_p + (double)lo * (from_p * (1.0 / 1073741824.0));
}

// TMA descriptors of one problem's C: box[k] is 2^k rows x ITEM_COLS columns,
// tile[k] is 2^k rows x TW columns (k = 0..TMA_BOXES-1).
constexpr int TMA_BOXES = 6;
static_assert((1 << (TMA_BOXES - 1)) == STAGE_ROWS, "boxes must compose any stage height");
struct TmaMaps {
    CUtensorMap box[TMA_BOXES];
    CUtensorMap tile[TMA_BOXES];
};
// -------------------------------------------------------------- kernel args
struct EvalArgs {
    TmaMaps tm0;                // one problem (inline_maps): its maps in the kernel's parameters
    ProbDesc pd0;               //   and its descriptor
    int32_t inline_maps;        // 1: use tm0, pd0 (parameter space: no fetch from global memory)
    const ProbDesc* probs;      // [nprob]
    const CUtensorMap* maps;    // [nprob][2 * TMA_BOXES] (box[], then tile[]); 64-byte aligned
    int32_t m, n, L, ntiles, nitems;
    int32_t fx_m, fx_n;         // rows of the tallest problem, columns of the widest (fixed-point bounds)
    const float4* rowA;  // sorted rows: (alpha hi, alpha lo, bound_up(alpha hi), 0)
    const int4* rowg;    // sorted rows: (group, first row, end row of the group, 0)
    const float2* B2;    // columns padded to padded_cols(n): (hi, lo) split of beta
    EvalCtl* ctl;
    int* err;            // error word (0 = ok)
    int32_t nlist;       // entries of desc
    const ItemDesc* desc;
    const int32_t* stage_row0;    // stage boundaries (ItemDesc::st0)
    const uint8_t* item_active;   // per item id: 1 if it has a unit to evaluate (screened), else NULL
    const uint32_t* unit_need;    // L x unit_words bitmask of units to evaluate, NULL = all
    const uint8_t* stage_m8;      // screened: [nstages][STAGE_ROWS] per row, bit w = tile w of its item needed
    uint32_t* stage_need;         // screened: bit s of word s / 32 set when stage s has a needed row
    unsigned long long* c_streamed; // NULL, or a counter: bytes of C the copies brought in (screened)
    int32_t unit_words;           // ceil(ntiles / 32)
    unsigned long long* rowfx;    // [m] fixed-point row sums of T (zeroed by the preparation kernel)
    unsigned long long* colfx;    // [n] fixed-point column sums of T
    unsigned long long* psix;  // [nprob][2]: psi of the exact-sum kernel's blocks (fixed point, hi, lo)
    XEntry* xent;      // flagged block sets of classes of at most XTALL_ROWS rows (capacity xent_cap)
    XEntry* xtall;     // those of taller classes (capacity xtall_cap)
    int32_t xent_cap, xtall_cap;
    float thr_flag;    // RD(theta^2 (1 - 2^-21)): a block whose FP32 bound stays at or below it has s = 0
    unsigned long long* fcount;  // NULL, or a counter of the flagged blocks (statistics)
    int32_t use_ct;    // 1: every problem has its transposed copy (ProbDesc::CT) for the exact sums
    uint32_t* xtmap;   // transposed route: per column task of a taller class, its set
    int32_t xtcol_cap;
    int32_t nprob;     // problems
    unsigned long long wait_ns;  // 0: the default limit of the evaluation kernel's waits; else this one
    int32_t stall;     // test hook: the consumer warps do not release stages (the waits run out)
    float* split_part; // [slots][ITEM_COLS][SPLIT_VALS]: a piece's (S', O) per column
    const SplitSet* sets;  // block sets of split groups
    int32_t nsets;
    const int* gate;   // NULL, or a device flag: 0 = skip this evaluation (batched solver trials)
    const int* prob_active;  // NULL, or per problem of a batch: 0 = its items are skipped
    const FxScale* pfx;      // NULL, or per problem of a batch: its fixed-point scale (from its own
                             // maxima and m, n); NULL: the scale of ctl's maxima with fx_m, fx_n
    float* zt;         // snapshot outputs (L x ntiles*TW) or NULL
    float* ot;
    // regularisation scalars
    float theta_hi, theta_lo;   // theta = mu*gamma as a float pair
    float th2_cut;              // S_hi below this: block surely below threshold
    float gamma;
    double inv2g;               // 1 / (2 gamma)
    float inv2g_hi, inv2g_lo;   // the same as a float pair
};

// Values per block of the reduction kernel's scratch (D's terms, the slope,
// the gradient's max norm).
constexpr int REDUCE_PARTS = 3;

struct ReduceArgs {
    int32_t m, n, nitems;
    int32_t fx_m, fx_n;
    const int32_t* perm;
    const uint8_t* item_active; // NULL = all items
    const unsigned long long* rowfx;
    const unsigned long long* colfx;
    const unsigned long long* psix;  // [2]: psi of the exact-sum kernel's blocks
    const EvalCtl* ctl;
    float gamma;
    const double* a_sorted;     // FP64 [m] sorted order
    const double* b;            // FP64 [n]
    const double* alpha_sorted; // FP64 [m]
    const double* beta;         // FP64 [n]
    // outputs (any may be NULL)
    double* out_caller;   // [1 + m + n]: D, dD/dalpha (caller order), dD/dbeta
    double* G_sorted;     // [m + n] minus gradient (sorted rows, then columns)
    const double* dir;    // [m + n] direction for dot(G, dir), or NULL
    double* scal;         // [4]: D, dot(G, dir), ||G||_inf, psi
    double* block_part;   // scratch [REDUCE_PARTS * nblocks]
    unsigned int* counter;// scratch, zero on entry, reset by the last block
    const int* err;       // evaluation error word: non-zero makes D NaN
    const int* gate;      // NULL, or a device flag: 0 = skip (batched solver trials)
};

// A block set for the exact-sum kernels (all lanes of the calling warp; lane
// 0 records it): rows [gstart, gend) of group l x the columns colg0 + k, k in
// mask.  With the transposed copy, a taller class's set also gets a column
// task per column (capacities hold every (group, column) once).
__device__ __forceinline__ void add_xentry(const EvalArgs& A, int gstart, int gend, int colg0, int prob, int l,
                                           uint32_t mask, int lane)
{
    const bool tall = gend - gstart > XTALL_ROWS;
    const int nc = __popc(mask);
    int e = 0, tb = 0;
    if (lane == 0) {
        e = atomicAdd(tall ? &A.ctl->nxtall : &A.ctl->nxent, 1);
        if (tall && A.use_ct) tb = atomicAdd(&A.ctl->ntcol, nc);
        if (A.fcount) atomicAdd(A.fcount, (unsigned long long)nc);
    }
    e = __shfl_sync(0xffffffffu, e, 0);
    tb = __shfl_sync(0xffffffffu, tb, 0);
    if (e >= (tall ? A.xtall_cap : A.xent_cap) || (tall && A.use_ct && tb + nc > A.xtcol_cap)) {
        if (lane == 0) atomicOr(A.err, 4);  // the capacities hold every (group, column) once: not reached
        return;
    }
    if (lane == 0) {
        XEntry& x = (tall ? A.xtall : A.xent)[e];
        x.gstart = gstart;
        x.gend = gend;
        x.colg0 = colg0;
        x.prob = prob;
        x.l = l;
        x.mask = mask;
        x.tbase = tb;
    }
    if (tall && A.use_ct && lane < nc) A.xtmap[tb + lane] = (uint32_t)e;
}

// launchers (otgs_eval.cu)
// Zeroes ctl, then writes rowA, B2 (and alpha_s_out), zeroes rowfx and
// colfx and records max [alpha hi]_+, max [beta hi]_+ in ctl.
void launch_prep(const double* alpha, bool alpha_sorted, const int32_t* perm, const double* beta,
                 int32_t m, int32_t n, float4* rowA, float2* B2, double* alpha_s_out,
                 unsigned long long* rowfx, unsigned long long* colfx, EvalCtl* ctl, cudaStream_t st);
// Encodes the maps for C (m x n, row stride ldc floats); "" on success.
std::string make_tmaps(const float* C, int64_t ldc, int64_t m, int64_t n, TmaMaps& T);
// evaluation kernel (otgs_stream.cu): persistent, n_ctas CTAs; a.ctl zeroed by launch_prep
void launch_stream(const EvalArgs& a, int n_ctas, cudaStream_t st);
// sets the evaluation kernel's shared-memory limit (once per device, before launches or capture)
bool stream_prepare();
// stage-mask kernel (otgs_stream.cu), screened evaluations: fills
// a.stage_m8 from a.unit_need for the active items.  Launch before launch_stream.
void launch_stage_masks(const EvalArgs& a, int n_sm, cudaStream_t st);
// split-finish kernel (otgs_stream.cu): adds the pieces' partial sums of the
// split groups' blocks and finishes them.  Launch right after launch_stream.
void launch_split_finish(const EvalArgs& a, cudaStream_t st);
// exact-sum kernel (otgs_stream.cu): the exact sums, Eq. 5 and the row sums
// of the blocks the evaluation kernel and the split-finish kernel flagged.
// Launch after the split-finish kernel with the same arguments.
void launch_exact(const EvalArgs& a, int n_sm, cudaStream_t st);
// Capacities of the flagged-block lists (host): one entry per (non-empty
// group, 32-column tile of its problem), each recorded at most once per
// evaluation; groups of at most XTALL_ROWS rows, and taller ones.
void exact_caps(const HostPlan& hp, int64_t& xent, int64_t& xtall, int64_t& tcols);
size_t stream_smem_bytes();
void launch_reduce(const ReduceArgs& a, cudaStream_t st);
int reduce_blocks(int32_t m, int32_t n);
// Cs row r = C row perm[r] - base (columns [0, n), zero up to ldcs).
void launch_transpose(const float* C, int64_t ldc, int32_t m, int32_t n, float* CT, int64_t ldct, cudaStream_t st);
void launch_gather_rows(const float* C, int64_t ldc, const int32_t* perm, int32_t base, int32_t m, int32_t n,
                        float* Cs, int64_t ldcs, cudaStream_t st);
void launch_permute_f64(const double* src, const int32_t* perm, int32_t m, double* dst,
                        bool to_sorted, cudaStream_t st);
void launch_check_finite(const float* C, int64_t ldc, int32_t m, int32_t n, const double* a,
                         const double* b, double* sums, int* flags, cudaStream_t st);

}  // namespace otgs
