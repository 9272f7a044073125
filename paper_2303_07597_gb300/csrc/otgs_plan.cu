// otgs_plan.cu -- host-side work decomposition over class groups.
//
// The dual's work splits into blocks (l, j): the rows of class l against
// target column j (Sec. 2.3, O(|L| n g) per evaluation).  On the GPU, rows are
// visited in class-sorted order, so every group is a contiguous range of
// sorted rows.  Consecutive groups are packed into panels (row ranges of
// whole groups, up to a panel height; a group taller than the split height is
// cut into pieces of that height, each a panel), and a work item is (panel,
// column chunk of ITEM_COLS columns).  Inside an item, each column's blocks are
// evaluated by one thread walking down the rows, so no block is split between
// threads (a tall group's pieces are added by a second kernel); items are
// handed out largest first.
//
// A batch of independent problems is planned as one block-diagonal problem:
// rows and columns are the concatenation of the problems', groups are
// (problem, class), and items only pair a problem's rows with its own columns.
#include <algorithm>
#include <cstring>
#include <numeric>

#include "otgs_internal.cuh"

namespace otgs {

std::string build_plan_batch(int32_t nprob, const int32_t* const* labels, const int64_t* pm, const int64_t* pn,
                             const int32_t* pL, const PlanParams& pp, HostPlan& hp)
{
    if (nprob <= 0) return "need at least one problem";
    hp = HostPlan();
    hp.nprob = nprob;
    int64_t m = 0, n = 0, L = 0, nb = 0;
    for (int32_t k = 0; k < nprob; k++) {
        if (pm[k] <= 0 || pn[k] <= 0 || pL[k] <= 0) return "m, n and L must be positive";
        if (!labels[k]) return "NULL labels";
        hp.proff.push_back((int32_t)m);
        hp.pcoff.push_back((int32_t)n);
        hp.pbcoff.push_back((int32_t)nb);
        hp.ploff.push_back((int32_t)L);
        hp.pm.push_back((int32_t)std::min<int64_t>(pm[k], INT32_MAX));
        hp.pn.push_back((int32_t)std::min<int64_t>(pn[k], INT32_MAX));
        m += pm[k];
        n += pn[k];
        nb += (pn[k] + 3) / 4 * 4;
        L += pL[k];
        hp.max_m = std::max<int64_t>(hp.max_m, pm[k]);
        hp.max_n = std::max<int64_t>(hp.max_n, pn[k]);
        if (m > INT32_MAX / 2 || n > INT32_MAX / 2 || L > INT32_MAX / 2) return "m, n and L must be below 2^30";
    }
    hp.m = m; hp.n = n; hp.L = (int32_t)L;
    // the bulk copy of a problem's last column chunk reads up to ITEM_COLS
    // entries from the chunk's start
    hp.nb2 = nprob == 1 ? padded_cols(n) : nb + ITEM_COLS;
    hp.ntiles = (int32_t)((n + TW - 1) / TW);
    // groups: (problem, class) -> global group ploff[k] + label
    std::vector<int64_t> cnt(L + 1, 0);
    for (int32_t k = 0; k < nprob; k++)
        for (int64_t i = 0; i < pm[k]; i++) {
            const int32_t lab = labels[k][i];
            if (lab < 0 || lab >= pL[k]) return "label out of range [0, L)";
            cnt[hp.ploff[k] + lab + 1]++;
            if (i > 0 && lab < labels[k][i - 1]) hp.sorted_identity = false;
        }
    hp.goff.assign(L + 1, 0);
    for (int64_t l = 0; l < L; l++) {
        hp.goff[l + 1] = hp.goff[l] + (int32_t)cnt[l + 1];
        hp.max_group = std::max<int32_t>(hp.max_group, (int32_t)cnt[l + 1]);
    }
    hp.gprob.resize(L);
    for (int32_t k = 0; k < nprob; k++)
        for (int32_t l = 0; l < pL[k]; l++) hp.gprob[hp.ploff[k] + l] = k;
    hp.perm.resize(m);
    hp.rgroup.resize(m);
    {
        std::vector<int32_t> fill(hp.goff.begin(), hp.goff.end() - 1);
        for (int32_t k = 0; k < nprob; k++)
            for (int64_t i = 0; i < pm[k]; i++) hp.perm[fill[hp.ploff[k] + labels[k][i]]++] = (int32_t)(hp.proff[k] + i);
    }
    hp.rowg.resize(m);
    for (int64_t l = 0; l < L; l++)
        for (int32_t r = hp.goff[l]; r < hp.goff[l + 1]; r++) {
            hp.rgroup[r] = (int32_t)l;
            hp.rowg[r] = make_int4((int32_t)l, hp.goff[l], hp.goff[l + 1], hp.gprob[l]);
        }

    // panels: runs of consecutive non-empty groups of one problem, closed
    // before they would exceed the panel height; tall groups in pieces
    int64_t pairs = 0;  // (row, column chunk) pairs of the problems
    for (int32_t k = 0; k < nprob; k++) pairs += row_chunks(pm[k], hp.pn[k]);
    const int32_t PANEL_ROWS = pp.panel_rows > 0 ? pp.panel_rows : panel_rows_for(pairs);
    const int32_t SPLIT = pp.split_rows > 0 ? pp.split_rows : SPLIT_ROWS;
    hp.panel_height = PANEL_ROWS;
    hp.split_height = SPLIT;
    hp.stage_fill = pp.stage_fill;
    hp.gpanel.assign(L, -1);
    int32_t cur0 = -1, cur_rows = 0, cur_prob = 0;
    int64_t slots = 0;
    auto nch_of = [&](int32_t k) { return (int32_t)((hp.pn[k] + ITEM_COLS - 1) / ITEM_COLS); };
    auto flush = [&]() {
        if (cur_rows == 0) return;
        hp.prow0.push_back(cur0);
        hp.prows.push_back(cur_rows);
        hp.pprob.push_back(cur_prob);
        hp.psplit.push_back(1);
        hp.psub.push_back(0);
        hp.pslot.push_back(-1);
        cur_rows = 0;
    };
    for (int32_t k = 0; k < nprob; k++) {
        for (int32_t l = hp.ploff[k]; l < hp.ploff[k] + pL[k]; l++) {
            const int32_t g = hp.goff[l + 1] - hp.goff[l];
            if (g == 0) continue;
            if (g > SPLIT) {
                // a tall group: panels of SPLIT rows of its own
                flush();
                hp.gpanel[l] = hp.npanels();
                const int32_t pieces = (g + SPLIT - 1) / SPLIT;
                for (int32_t q = 0; q < pieces; q++) {
                    hp.prow0.push_back(hp.goff[l] + q * SPLIT);
                    hp.prows.push_back(std::min(SPLIT, g - q * SPLIT));
                    hp.pprob.push_back(k);
                    hp.psplit.push_back(pieces);
                    hp.psub.push_back(q);
                    hp.pslot.push_back((int32_t)slots);
                }
                slots += (int64_t)pieces * nch_of(k);
                continue;
            }
            if (cur_rows > 0 && cur_rows + g > PANEL_ROWS) flush();
            if (cur_rows == 0) {
                cur0 = hp.goff[l];
                cur_prob = k;
            }
            hp.gpanel[l] = hp.npanels();
            cur_rows += g;
            if (cur_rows >= PANEL_ROWS) flush();
        }
        flush();  // panels never span two problems
    }
    if (slots > INT32_MAX / (ITEM_COLS * SPLIT_VALS)) return "too many pieces of tall groups";
    hp.nsplit_slots = slots;

    // stages of each panel
    const int np = hp.npanels();
    hp.pst0.resize(np);
    hp.pnst.resize(np);
    for (int p = 0; p < np; p++) {
        hp.pst0[p] = (int32_t)hp.stage_row0.size();
        const int32_t end = hp.prow0[p] + hp.prows[p];
        int32_t ra = hp.prow0[p], cnt = 0;
        while (ra < end) {
            hp.stage_row0.push_back(ra);
            cnt++;
            int32_t nr = std::min<int32_t>(STAGE_ROWS, end - ra);
            if (pp.stage_fill > 0 && ra + nr < end && hp.psplit[p] == 1) {
                // the group holding the stage's last row: does it go on past the stage?
                const int32_t l = hp.rgroup[ra + nr - 1], gs = hp.goff[l], ge = hp.goff[l + 1];
                if (ge > ra + nr && ge - gs <= STAGE_ROWS && gs > ra && gs - ra >= pp.stage_fill) nr = gs - ra;
            }
            ra += nr;
        }
        hp.stage_row0.push_back(end);
        hp.pnst[p] = cnt;
    }
    if (hp.stage_row0.size() > (size_t)INT32_MAX / 2) return "too many stages";

    // work items: (panel, column chunk of its problem)
    hp.pW.assign(np, ITEM_COLS);
    hp.pnch.resize(np);
    hp.pitem.resize(np);
    std::vector<double> cost;
    for (int p = 0; p < np; p++) {
        const int32_t k = hp.pprob[p], nch = nch_of(k);
        hp.pnch[p] = nch;
        hp.pitem[p] = hp.nitems();
        for (int32_t c = 0; c < nch; c++) {
            hp.item_panel.push_back(p);
            hp.item_chunk.push_back(c);
            const int64_t cols = std::min<int64_t>(ITEM_COLS, hp.pn[k] - (int64_t)c * ITEM_COLS);
            cost.push_back((double)hp.prows[p] * (double)cols);
        }
    }
    hp.exec_order.resize(hp.nitems());
    std::iota(hp.exec_order.begin(), hp.exec_order.end(), 0);
    std::stable_sort(hp.exec_order.begin(), hp.exec_order.end(),
                     [&](int32_t x, int32_t y) { return cost[x] > cost[y]; });
    hp.desc.resize(hp.nitems());
    hp.nstages = 0;
    for (int q = 0; q < hp.nitems(); q++) {
        const int32_t item = hp.exec_order[q];
        const int32_t p = hp.item_panel[item], cc = hp.item_chunk[item], k = hp.pprob[p];
        ItemDesc d;
        memset(&d, 0, sizeof(d));
        d.item = item;
        d.p = p;
        d.r0 = hp.prow0[p];
        d.rows = hp.prows[p];
        d.col0 = cc * ITEM_COLS;
        d.ncols = (int)std::min<int64_t>(ITEM_COLS, hp.pn[k] - (int64_t)d.col0);
        d.nst = hp.pnst[p];
        d.st0 = hp.pst0[p];
        d.sbase = (int)hp.nstages;
        d.split = hp.psplit[p];
        d.sub = hp.psub[p];
        // slots of the set (group, chunk cc): pslot + cc * split + [0, split)
        d.part = d.split > 1 ? hp.pslot[p] + cc * d.split : -1;
        d.prob = k;
        hp.nstages += d.nst;
        hp.desc[q] = d;
    }
    if (hp.nstages > INT32_MAX / STAGE_ROWS) return "m x n too large for the stage tables";
    // block sets of the split groups: (group, chunk)
    for (int p = 0; p < np; p++) {
        if (hp.psplit[p] == 1 || hp.psub[p] != 0) continue;
        const int32_t l = hp.rgroup[hp.prow0[p]], k = hp.pprob[p];
        for (int32_t cc = 0; cc < nch_of(k); cc++) {
            SplitSet s;
            s.l = l;
            s.col0 = cc * ITEM_COLS;
            s.split = hp.psplit[p];
            s.part = hp.pslot[p] + cc * s.split;
            s.item0 = hp.pitem[p] + cc;
            s.rstart = hp.goff[l];
            s.rend = hp.goff[l + 1];
            s.prob = k;
            hp.sets.push_back(s);
        }
    }
    return "";
}

std::string build_plan(const int32_t* labels, int64_t m, int64_t n, int32_t L, HostPlan& hp)
{
    return build_plan_batch(1, &labels, &m, &n, &L, PlanParams(), hp);
}

}  // namespace otgs
