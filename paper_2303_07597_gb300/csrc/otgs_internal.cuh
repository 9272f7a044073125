// otgs_internal.cuh -- shared declarations of the CUDA path (not part of the ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "otgs.h"

namespace otgs {

// ---------------------------------------------------------------- geometry
// A "unit" is (group l, tile of TW consecutive target columns): g_l rows of C
// by TW columns, one 128-byte line per row.  A warp reads a unit four rows
// at a time, eight lanes per row, one float4 per lane.
constexpr int TW = 32;
constexpr int NWARPS = 8;
constexpr int NTHREADS = NWARPS * 32;
// The evaluation kernel streams C through shared-memory stages of STAGE_ROWS
// rows x STAGE_COLS columns (two tiles; 256-byte rows keep the TMA engine at
// full rate).  Groups of at most SMALL_MAX_ROWS rows are packed into "small"
// panels (one stage per tile pair; each consumer warp owns a contiguous range
// of whole groups); larger groups form a "big" panel of their own
// (ceil(g / STAGE_ROWS) stages per tile pair, rows split over the warps).
constexpr int STAGE_ROWS = 128;
constexpr int STAGE_COLS = 2 * TW;
constexpr int NSTAGES = 5;
constexpr int SMALL_MAX_ROWS = STAGE_ROWS;
constexpr int PANEL_ROWS = STAGE_ROWS;  // row budget of a small panel
constexpr int PANEL_MAX_GROUPS = 64;    // group budget of a small panel
constexpr int SMALL_CHUNK = 256;        // columns per small-panel work item (multiple of STAGE_COLS)
constexpr int BIG_MAX_CHUNK = 256;      // columns per big-panel work item (max, multiple of STAGE_COLS)
constexpr int BIG_SMEM_ROWS = 4096;     // big groups up to this size sum rows in shared memory
constexpr double ITEM_BYTES = 2.0 * (1 << 20);  // target C bytes per big-panel item

// Columns of the float-pair split of beta, padded to whole stages.
inline int32_t padded_cols(int32_t ntiles) { return (ntiles + 1) / 2 * STAGE_COLS; }

// alpha_i (resp. beta_j) rounded up by a relative 2^-22: c_ij < A'_i + B'_j
// (FP32, round to nearest) holds whenever alpha_i + beta_j - c_ij > 0, so the
// test rejects only elements whose f is certainly <= 0.
__device__ __forceinline__ float bound_up(float h) { return __fadd_ru(h, __fmul_ru(fabsf(h), 0x1p-22f)); }

// A work item as the evaluation kernel sees it, in execution order (128 B).
struct ItemDesc {
    int item, p, cc, kind;   // item id, panel, column chunk, 0 small / 1 big panel
    int W, rows, r0, l;      // columns per item; panel (small) or group (big) rows; first sorted row; group (big)
    int nst, nt, t0, ncols;  // stages per tile (big), tiles, first tile, columns of this item
    int rb_lo, rb_hi, col0, ngroups;  // row-partial base (int64 halves), first column, groups of the panel
    int pw[NWARPS + 1];      // first pginfo entry of each consumer warp (small panels), then the end
    int pad[7];
};

// ------------------------------------------------------------------ host plan
// Built once from the labels at create.  "Sorted" row r is the r-th row in
// (label, caller index) order; groups are contiguous ranges of sorted rows.
struct HostPlan {
    int64_t m = 0, n = 0;
    int32_t L = 0, ntiles = 0;
    std::vector<int32_t> perm;    // sorted r -> caller row
    std::vector<int32_t> goff;    // L+1 offsets (sorted rows)
    std::vector<int32_t> rgroup;  // sorted r -> group
    // panels
    std::vector<int32_t> pkind;   // 0 small, 1 big
    std::vector<int32_t> prows;   // rows of the panel
    std::vector<int32_t> pW;      // columns per work item (multiple of TW)
    std::vector<int32_t> pnch;    // work items (column chunks) of the panel
    std::vector<int64_t> prp;     // base of the panel's row partials
    std::vector<int32_t> pitem;   // first work-item id of the panel
    std::vector<int32_t> pw_off;  // [npanels * NWARPS + 1] offsets into pgrp
    std::vector<int32_t> pgrp;    // groups of each (panel, warp), LPT-balanced
    std::vector<int32_t> gpanel;  // group -> panel (-1 for empty groups)
    std::vector<int32_t> gsrow;   // group -> first local row in its panel
    std::vector<int32_t> prow0;   // first sorted row of the panel (rows are contiguous)
    std::vector<int4> pginfo;     // per pgrp entry: {group, first sorted row, rows, row in panel}
    std::vector<ItemDesc> desc;   // work items in execution order
    // work items, id = pitem[p] + chunk
    std::vector<int32_t> item_panel, item_chunk;
    std::vector<int32_t> exec_order;  // item ids, largest first
    int64_t rowpart_len = 0;
    bool sorted_identity = true;  // labels already non-decreasing
    int npanels() const { return (int)pkind.size(); }
    int nitems() const { return (int)item_panel.size(); }
};

// Returns an empty string on success, else an error message.
std::string build_plan(const int32_t* labels, int64_t m, int64_t n, int32_t L, HostPlan& hp);

// ---------------------------------------------------------------- device plan
struct DevPlan {
    int32_t *perm, *goff, *rgroup;
    int32_t *pkind, *prows, *pW, *pnch, *pitem, *pw_off, *pgrp, *gpanel, *gsrow;
    int64_t *prp;
    int32_t *item_panel, *item_chunk, *exec_order;
    int32_t *prow0;
    int4 *pginfo;
    ItemDesc *desc;
};

// -------------------------------------------------------------- kernel args
struct EvalArgs {
    const float* C;
    int64_t ldc;
    int32_t m, n, L, ntiles, npanels, nitems;
    const float2* A2;  // sorted rows: (hi, lo) split of alpha, padded by 2 (copied in 16-byte blocks)
    const float2* B2;  // columns padded to padded_cols(ntiles): (hi, lo) split of beta
    const float* Bp;   // bound_up(beta hi) per column, -inf in the padding
    int* work;         // work-item counter, zero at launch
    int* err;          // error word (0 = ok)
    int32_t nlist;     // entries of items
    DevPlan plan;
    const int32_t* items;         // item ids, one per CTA
    const uint8_t* item_active;   // per item id: 1 if launched (its partials valid)
    const uint32_t* unit_need;    // L x unit_words bitmask of units to stream, NULL = all
    int32_t unit_words;           // ceil(ntiles / 32)
    double* rowpart;
    double* colpart;   // npanels x n
    double* psipart;   // per item id
    float* zt;         // snapshot outputs (L x ntiles*TW) or NULL
    float* ot;
    // regularisation scalars
    float theta_hi, theta_lo;   // theta = mu*gamma as a float pair
    float th2_cut;              // S_hi below this: block surely below threshold
    float gamma;
    double inv2g;               // 1 / (2 gamma)
    unsigned long long* units_done;  // counter of streamed units (may be NULL)
};

struct ReduceArgs {
    int32_t m, n, npanels, nitems;
    DevPlan plan;
    const uint8_t* item_active;
    const double* rowpart;
    const double* colpart;
    const double* psipart;
    const double* a_sorted;     // FP64 [m] sorted order
    const double* b;            // FP64 [n]
    const double* alpha_sorted; // FP64 [m]
    const double* beta;         // FP64 [n]
    // outputs (any may be NULL)
    double* out_caller;   // [1 + m + n]: D, dD/dalpha (caller order), dD/dbeta
    double* G_sorted;     // [m + n] minus gradient (sorted rows, then columns)
    const double* dir;    // [m + n] direction for dot(G, dir), or NULL
    double* scal;         // [4]: D, dot(G, dir), ||G||_inf, psi
    double* block_part;   // scratch [3 * nblocks]
    unsigned int* counter;// scratch, zero on entry, reset by the last block
    const int* err;       // evaluation error word: non-zero makes D NaN
};

// launchers (otgs_eval.cu)
void launch_prep(const double* alpha, bool alpha_sorted, const int32_t* perm, const double* beta,
                 int32_t m, int32_t n, int32_t ntiles, float2* A2, float2* B2, float* Bp,
                 double* alpha_s_out, cudaStream_t st);
// TMA descriptors of C: box k is 2^k rows x STAGE_COLS columns (k = 0..TMA_BOXES-1).
constexpr int TMA_BOXES = 8;
struct TmaMaps {
    CUtensorMap box[TMA_BOXES];
};
// Encodes the maps for C (m x n, row stride ldc floats); "" on success.
std::string make_tmaps(const float* C, int64_t ldc, int64_t m, int64_t n, TmaMaps& T);
// evaluation kernel (otgs_stream.cu): persistent, n_ctas CTAs; a.work must be zero
void launch_stream(const EvalArgs& a, const TmaMaps& T, int n_ctas, cudaStream_t st);
size_t stream_smem_bytes();
void launch_reduce(const ReduceArgs& a, cudaStream_t st);
int reduce_blocks(int32_t m, int32_t n);
void launch_gather_rows(const float* C, int64_t ldc, const int32_t* perm, int32_t m, int32_t n,
                        float* Cs, int64_t ldcs, cudaStream_t st);
void launch_permute_f64(const double* src, const int32_t* perm, int32_t m, double* dst,
                        bool to_sorted, cudaStream_t st);
void launch_check_finite(const float* C, int64_t ldc, int32_t m, int32_t n, const double* a,
                         const double* b, double* sums, int* flags, cudaStream_t st);

}  // namespace otgs
