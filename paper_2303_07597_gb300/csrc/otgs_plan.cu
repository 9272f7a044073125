// otgs_plan.cu -- host-side work decomposition over class groups.
//
// The dual's work splits into blocks (l, j): the rows of class l against
// target column j (Sec. 2.3, O(|L| n g) per evaluation).  On the GPU, rows are
// visited in class-sorted order and columns in tiles of TW, so the unit of
// work is (group, tile).  Units are gathered into work items:
//   small panel: consecutive small groups (<= SMALL_MAX_ROWS rows each), up to
//                PANEL_ROWS rows, each consumer warp owning a contiguous run of
//                whole groups, times SMALL_CHUNK columns; its rows are one
//                contiguous range of sorted rows, kept in that order in
//                shared memory;
//   big panel:   one large group whose rows are split over all consumer warps,
//                times a column chunk of about ITEM_BYTES of C.
// Every row of a panel accumulates its row sum per item into the row-partial
// buffer; the reduction kernel adds them in a fixed order.
#include <algorithm>
#include <cstring>
#include <numeric>

#include "otgs_internal.cuh"

namespace otgs {

std::string build_plan(const int32_t* labels, int64_t m, int64_t n, int32_t L, HostPlan& hp)
{
    if (m <= 0 || n <= 0 || L <= 0) return "m, n and L must be positive";
    if (m > INT32_MAX / 2 || n > INT32_MAX / 2) return "m and n must be below 2^30";
    hp = HostPlan();
    hp.m = m; hp.n = n; hp.L = L;
    hp.ntiles = (int32_t)((n + TW - 1) / TW);
    std::vector<int64_t> cnt(L + 1, 0);
    for (int64_t i = 0; i < m; i++) {
        if (labels[i] < 0 || labels[i] >= L) return "label out of range [0, L)";
        cnt[labels[i] + 1]++;
        if (i > 0 && labels[i] < labels[i - 1]) hp.sorted_identity = false;
    }
    hp.goff.assign(L + 1, 0);
    for (int32_t l = 0; l < L; l++) hp.goff[l + 1] = hp.goff[l] + (int32_t)cnt[l + 1];
    hp.perm.resize(m);
    hp.rgroup.resize(m);
    {
        std::vector<int32_t> fill(hp.goff.begin(), hp.goff.end() - 1);
        for (int64_t i = 0; i < m; i++) hp.perm[fill[labels[i]]++] = (int32_t)i;
    }
    for (int32_t l = 0; l < L; l++)
        for (int32_t r = hp.goff[l]; r < hp.goff[l + 1]; r++) hp.rgroup[r] = l;

    hp.gpanel.assign(L, -1);
    hp.gsrow.assign(L, 0);
    hp.pw_off.push_back(0);
    auto gsize = [&](int32_t l) { return hp.goff[l + 1] - hp.goff[l]; };

    // small panels: runs of consecutive small groups in label order (a big or
    // empty-free boundary closes the panel, so its rows are one contiguous
    // range of sorted rows, loadable by TMA boxes)
    std::vector<int32_t> cur;
    int32_t cur_rows = 0;
    auto flush_small = [&]() {
        if (cur.empty()) return;
        int p = hp.npanels();
        hp.pkind.push_back(0);
        hp.prows.push_back(cur_rows);
        hp.prow0.push_back(hp.goff[cur.front()]);
        hp.pW.push_back(SMALL_CHUNK);
        // each consumer warp takes a contiguous run of whole groups, the runs
        // split where the cumulative row count crosses multiples of rows / 8
        int w = 0;
        int32_t cum = 0;
        hp.pgrp.insert(hp.pgrp.end(), cur.begin(), cur.end());
        const int32_t base = (int32_t)hp.pgrp.size() - (int32_t)cur.size();
        std::vector<int32_t> first(NWARPS + 1, (int32_t)cur.size());
        first[0] = 0;
        for (size_t k = 0; k < cur.size(); k++) {
            const int32_t l = cur[k];
            const int32_t g = gsize(l);
            while (w + 1 < NWARPS && 2 * (cum + g / 2) > 2 * ((int64_t)(w + 1) * cur_rows / NWARPS)) {
                w++;
                first[w] = (int32_t)k;
            }
            cum += g;
            hp.gpanel[l] = p;
            hp.gsrow[l] = hp.goff[l] - hp.goff[cur.front()];  // rows stay in sorted order
        }
        for (int v = w + 1; v <= NWARPS; v++) first[v] = (int32_t)cur.size();
        for (int v = 1; v <= NWARPS; v++) hp.pw_off.push_back(base + first[v]);
        cur.clear();
        cur_rows = 0;
    };
    for (int32_t l = 0; l < L; l++) {
        int32_t g = gsize(l);
        if (g == 0) continue;
        if (g > SMALL_MAX_ROWS) {
            flush_small();
            continue;
        }
        if (cur_rows + g > PANEL_ROWS || (int)cur.size() >= PANEL_MAX_GROUPS) flush_small();
        cur.push_back(l);
        cur_rows += g;
    }
    flush_small();
    // big panels: one group each, all warps
    for (int32_t l = 0; l < L; l++) {
        int32_t g = gsize(l);
        if (g <= SMALL_MAX_ROWS) continue;
        int p = hp.npanels();
        hp.pkind.push_back(1);
        hp.prows.push_back(g);
        hp.prow0.push_back(hp.goff[l]);
        int64_t w = (int64_t)(ITEM_BYTES / (4.0 * g));
        w = (w / STAGE_COLS) * STAGE_COLS;
        w = std::max<int64_t>(STAGE_COLS, std::min<int64_t>(BIG_MAX_CHUNK, w));
        hp.pW.push_back((int32_t)w);
        hp.pgrp.push_back(l);
        hp.gpanel[l] = p;
        hp.gsrow[l] = 0;
        for (int k = 0; k < NWARPS; k++) hp.pw_off.push_back((int32_t)hp.pgrp.size());
    }
    // work items and row-partial layout
    int np = hp.npanels();
    hp.pnch.resize(np);
    hp.prp.resize(np);
    hp.pitem.resize(np);
    int64_t rp = 0;
    std::vector<double> cost;
    for (int p = 0; p < np; p++) {
        int32_t W = hp.pW[p];
        int32_t nch = (int32_t)((n + W - 1) / W);
        hp.pnch[p] = nch;
        hp.prp[p] = rp;
        rp += (int64_t)nch * hp.prows[p];
        hp.pitem[p] = hp.nitems();
        for (int32_t c = 0; c < nch; c++) {
            hp.item_panel.push_back(p);
            hp.item_chunk.push_back(c);
            int64_t cols = std::min<int64_t>(W, n - (int64_t)c * W);
            cost.push_back((double)hp.prows[p] * (double)cols);
        }
    }
    hp.rowpart_len = rp;
    hp.exec_order.resize(hp.nitems());
    std::iota(hp.exec_order.begin(), hp.exec_order.end(), 0);
    std::stable_sort(hp.exec_order.begin(), hp.exec_order.end(),
                     [&](int32_t x, int32_t y) { return cost[x] > cost[y]; });
    hp.pginfo.resize(hp.pgrp.size());
    for (size_t k = 0; k < hp.pgrp.size(); k++) {
        const int32_t l = hp.pgrp[k];
        hp.pginfo[k] = make_int4(l, hp.goff[l], hp.goff[l + 1] - hp.goff[l], hp.gsrow[l]);
    }
    hp.desc.resize(hp.nitems());
    for (int k = 0; k < hp.nitems(); k++) {
        const int32_t item = hp.exec_order[k];
        const int32_t p = hp.item_panel[item], cc = hp.item_chunk[item];
        ItemDesc d;
        memset(&d, 0, sizeof(d));
        d.item = item; d.p = p; d.cc = cc; d.kind = hp.pkind[p];
        d.W = hp.pW[p]; d.rows = hp.prows[p]; d.r0 = hp.prow0[p];
        d.l = d.kind ? hp.pgrp[hp.pw_off[p * NWARPS]] : -1;
        d.nst = d.kind ? (d.rows + STAGE_ROWS - 1) / STAGE_ROWS : 1;
        d.col0 = cc * d.W;
        d.ncols = (int)std::min<int64_t>(d.W, n - (int64_t)d.col0);
        d.nt = (d.ncols + TW - 1) / TW;
        d.t0 = d.col0 / TW;
        const int64_t rb = hp.prp[p] + (int64_t)cc * d.rows;
        d.rb_lo = (int)(rb & 0xffffffff);
        d.rb_hi = (int)(rb >> 32);
        d.ngroups = hp.pw_off[p * NWARPS + NWARPS] - hp.pw_off[p * NWARPS];
        for (int w = 0; w <= NWARPS; w++) d.pw[w] = hp.pw_off[p * NWARPS + w];
        hp.desc[k] = d;
    }
    return "";
}

}  // namespace otgs
