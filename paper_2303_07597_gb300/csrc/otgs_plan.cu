// otgs_plan.cu -- host-side work decomposition over class groups.
//
// The dual's work splits into blocks (l, j): the rows of class l against
// target column j (Sec. 2.3, O(|L| n g) per evaluation).  On the GPU, rows are
// visited in class-sorted order, so every group is a contiguous range of
// sorted rows.  Consecutive groups are packed into panels (row ranges of
// whole groups, up to panel_rows(m, n) rows; a group taller than SPLIT_ROWS is
// cut into pieces of SPLIT_ROWS rows, each a panel),
// and a work item is (panel, column chunk of ITEM_COLS columns).  Inside an
// item, each column's blocks are evaluated by one thread walking down the
// rows, so no block is ever split between threads; items are handed out
// largest first.
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
    for (int32_t l = 0; l < L; l++) {
        hp.goff[l + 1] = hp.goff[l] + (int32_t)cnt[l + 1];
        hp.max_group = std::max<int32_t>(hp.max_group, (int32_t)cnt[l + 1]);
    }
    hp.perm.resize(m);
    hp.rgroup.resize(m);
    {
        std::vector<int32_t> fill(hp.goff.begin(), hp.goff.end() - 1);
        for (int64_t i = 0; i < m; i++) hp.perm[fill[labels[i]]++] = (int32_t)i;
    }
    hp.rowg.resize(m);
    for (int32_t l = 0; l < L; l++)
        for (int32_t r = hp.goff[l]; r < hp.goff[l + 1]; r++) {
            hp.rgroup[r] = l;
            hp.rowg[r] = make_int4(l, hp.goff[l], hp.goff[l + 1], 0);
        }

    // panels: runs of consecutive non-empty groups in label order, closed
    // before they would exceed the panel height
    const int32_t PANEL_ROWS = panel_rows(m, n);
    hp.gpanel.assign(L, -1);
    int32_t cur0 = -1, cur_rows = 0, pieces_before = 0;
    auto flush = [&]() {
        if (cur_rows == 0) return;
        hp.prow0.push_back(cur0);
        hp.prows.push_back(cur_rows);
        hp.psplit.push_back(1);
        hp.psub.push_back(0);
        hp.pslot.push_back(-1);
        cur_rows = 0;
    };
    for (int32_t l = 0; l < L; l++) {
        const int32_t g = hp.goff[l + 1] - hp.goff[l];
        if (g == 0) continue;
        if (g > SPLIT_ROWS) {
            // a tall group: panels of SPLIT_ROWS rows of its own
            flush();
            hp.gpanel[l] = hp.npanels();
            const int32_t pieces = (g + SPLIT_ROWS - 1) / SPLIT_ROWS;
            for (int32_t k = 0; k < pieces; k++) {
                hp.prow0.push_back(hp.goff[l] + k * SPLIT_ROWS);
                hp.prows.push_back(std::min(SPLIT_ROWS, g - k * SPLIT_ROWS));
                hp.psplit.push_back(pieces);
                hp.psub.push_back(k);
                hp.pslot.push_back(pieces_before);
            }
            pieces_before += pieces;
            continue;
        }
        if (cur_rows > 0 && cur_rows + g > PANEL_ROWS) flush();
        if (cur_rows == 0) cur0 = hp.goff[l];
        hp.gpanel[l] = hp.npanels();
        cur_rows += g;
        if (cur_rows >= PANEL_ROWS) flush();
    }
    flush();

    // work items: (panel, column chunk)
    const int np = hp.npanels();
    const int32_t nch = (int32_t)((n + ITEM_COLS - 1) / ITEM_COLS);
    hp.pW.assign(np, ITEM_COLS);
    hp.pnch.assign(np, nch);
    hp.pitem.resize(np);
    std::vector<double> cost;
    for (int p = 0; p < np; p++) {
        hp.pitem[p] = hp.nitems();
        for (int32_t c = 0; c < nch; c++) {
            hp.item_panel.push_back(p);
            hp.item_chunk.push_back(c);
            const int64_t cols = std::min<int64_t>(ITEM_COLS, n - (int64_t)c * ITEM_COLS);
            cost.push_back((double)hp.prows[p] * (double)cols);
        }
    }
    hp.exec_order.resize(hp.nitems());
    std::iota(hp.exec_order.begin(), hp.exec_order.end(), 0);
    std::stable_sort(hp.exec_order.begin(), hp.exec_order.end(),
                     [&](int32_t x, int32_t y) { return cost[x] > cost[y]; });
    hp.desc.resize(hp.nitems());
    hp.nstages = 0;
    for (int k = 0; k < hp.nitems(); k++) {
        const int32_t item = hp.exec_order[k];
        const int32_t p = hp.item_panel[item], cc = hp.item_chunk[item];
        ItemDesc d;
        memset(&d, 0, sizeof(d));
        d.item = item;
        d.p = p;
        d.r0 = hp.prow0[p];
        d.rows = hp.prows[p];
        d.col0 = cc * ITEM_COLS;
        d.ncols = (int)std::min<int64_t>(ITEM_COLS, n - (int64_t)d.col0);
        d.nst = (d.rows + STAGE_ROWS - 1) / STAGE_ROWS;
        d.sbase = (int)hp.nstages;
        d.split = hp.psplit[p];
        d.sub = hp.psub[p];
        // slots of the set (group, chunk cc): pslot * nch + cc * split + [0, split)
        d.part = d.split > 1 ? hp.pslot[p] * nch + cc * d.split : -1;
        hp.nstages += d.nst;
        hp.desc[k] = d;
    }
    if (hp.nstages > INT32_MAX / STAGE_ROWS) return "m x n too large for the stage tables";
    hp.nsplit_slots = (int64_t)pieces_before * nch;
    // block sets of the split groups: (group, chunk)
    for (int p = 0; p < np; p++) {
        if (hp.psplit[p] == 1 || hp.psub[p] != 0) continue;
        const int32_t l = hp.rgroup[hp.prow0[p]];
        for (int32_t cc = 0; cc < nch; cc++) {
            SplitSet s;
            s.l = l;
            s.col0 = cc * ITEM_COLS;
            s.split = hp.psplit[p];
            s.part = hp.pslot[p] * nch + cc * s.split;
            s.item0 = hp.pitem[p] + cc;
            s.rstart = hp.goff[l];
            s.rend = hp.goff[l + 1];
            s.pad = 0;
            hp.sets.push_back(s);
        }
    }
    return "";
}

}  // namespace otgs
