// otgs_plan.cu -- host-side work decomposition over class groups.
//
// The dual's work splits into blocks (l, j): the rows of class l against
// target column j (Sec. 2.3, O(|L| n g) per evaluation).  On the GPU, rows are
// visited in class-sorted order and columns in tiles of TW, so the unit of
// work is (group, tile).  Units are gathered into work items (one CTA each):
//   small panel: consecutive small groups (<= SMALL_MAX_ROWS rows each), up to
//                PANEL_ROWS rows, each group owned by one warp (LPT balance),
//                times SMALL_CHUNK columns;
//   big panel:   one large group whose rows are split over all warps, times a
//                column chunk sized to about ITEM_BYTES of C.
// Every row of a panel accumulates its row sum per item into the row-partial
// buffer; the reduction kernel adds them in a fixed order.
#include <algorithm>
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

    // small panels: consecutive small groups in label order
    std::vector<int32_t> cur;
    int32_t cur_rows = 0;
    auto flush_small = [&]() {
        if (cur.empty()) return;
        int p = hp.npanels();
        hp.pkind.push_back(0);
        hp.prows.push_back(cur_rows);
        hp.pW.push_back(SMALL_CHUNK);
        // LPT: largest groups first, each to the least-loaded warp (cost in
        // 4-row steps plus one step of per-unit epilogue)
        std::vector<int32_t> ord(cur);
        std::stable_sort(ord.begin(), ord.end(),
                         [&](int32_t x, int32_t y) { return gsize(x) > gsize(y); });
        std::vector<std::vector<int32_t>> wg(NWARPS);
        std::vector<int64_t> load(NWARPS, 0);
        for (int32_t l : ord) {
            int w = (int)(std::min_element(load.begin(), load.end()) - load.begin());
            wg[w].push_back(l);
            load[w] += (gsize(l) + 3) / 4 + 1;
        }
        int32_t srow = 0;
        for (int w = 0; w < NWARPS; w++) {
            for (int32_t l : wg[w]) {
                hp.pgrp.push_back(l);
                hp.gpanel[l] = p;
                hp.gsrow[l] = srow;
                srow += gsize(l);
            }
            hp.pw_off.push_back((int32_t)hp.pgrp.size());
        }
        cur.clear();
        cur_rows = 0;
    };
    for (int32_t l = 0; l < L; l++) {
        int32_t g = gsize(l);
        if (g == 0 || g > SMALL_MAX_ROWS) continue;
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
        int64_t w = (int64_t)(ITEM_BYTES / (4.0 * g));
        w = (w / TW) * TW;
        w = std::max<int64_t>(TW, std::min<int64_t>(BIG_MAX_CHUNK, w));
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
    return "";
}

}  // namespace otgs
