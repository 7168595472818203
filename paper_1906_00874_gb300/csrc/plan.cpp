// Host planner: validation, block tree, arena layout and the expansion of the
// H-LU recursion (Sec. 3.1) into tasks grouped in dependency waves.
#include "plan.h"

#include <climits>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <new>
#include <condition_variable>
#include <map>
#include <mutex>
#include <system_error>
#include <thread>
#include <utility>
#include <functional>
#include <unordered_map>

#include "../../include/hlu.h"

namespace hlu {

static inline int64_t align8(int64_t x) { return (x + 7) & ~int64_t(7); }

Planner::~Planner() {
    for (Block *b : blocks_owned) delete b;
}

void Planner::release_work() {
    for (Block *b : blocks_owned) delete b;
    std::vector<Block *>().swap(blocks_owned);
    root = nullptr;
    std::vector<Obj>().swap(objs);
    std::vector<CellState>().swap(dep.cell);
    std::vector<int32_t>().swap(dep.pred_mark);
    std::vector<int32_t>().swap(dep.rpool_task);
    std::vector<int32_t>().swap(dep.rpool_next);
    std::vector<PlanItem>().swap(plan_items);
    std::vector<int32_t>().swap(dep.touch_obj);
    std::vector<int32_t>().swap(dep.touch_cell);
    std::vector<int32_t>().swap(dep.touch_task);
    std::vector<uint8_t>().swap(dep.touch_write);
    std::vector<std::array<int32_t, 4>>().swap(temp_shape);
    std::vector<int64_t>().swap(temp_size);
    std::vector<int32_t>().swap(dep.temp_first);
    std::vector<int32_t>().swap(dep.temp_last);
    for (Plan *p : {&fplan, &splan, &mplan}) {  // the executors use the successor lists only
        std::vector<int32_t>().swap(p->pred_ptr);
        std::vector<int32_t>().swap(p->pred_idx);
    }
}

void Plan::release_tasks() {
    kind_count[K_GETRF] = (int64_t)getrf.size();
    kind_count[K_TRSM] = (int64_t)trsm.size();
    kind_count[K_PROJECT] = (int64_t)project.size();
    kind_count[K_ACCUM] = (int64_t)accum.size();
    kind_count[K_RADD] = (int64_t)radd.size();
    kind_count[K_SPLIT] = (int64_t)split.size();
    last_indeg = indeg.empty() ? 0 : indeg.back();
    std::vector<TGetrf>().swap(getrf);
    std::vector<TTrsm>().swap(trsm);
    std::vector<TProject>().swap(project);
    std::vector<TAccum>().swap(accum);
    std::vector<TRadd>().swap(radd);
    std::vector<TSplit>().swap(split);
    std::vector<Term>().swap(terms);
    std::vector<Piece>().swap(pieces);
    for (auto &w : wave) std::vector<int32_t>().swap(w);
    for (std::vector<int32_t> *v : {&task_code, &pred_ptr, &pred_idx, &succ_ptr, &succ_idx, &indeg, &roots})
        std::vector<int32_t>().swap(*v);
    std::vector<float>().swap(root_bl);
}

// ------------------------------------------------------------------ objects
int32_t Planner::new_obj(int32_t row_cl, int32_t col_cl, int32_t nr_if_none) {
    Obj o;
    o.row_cl = row_cl;
    o.col_cl = col_cl;
    o.nr = row_cl >= 0 ? cl[row_cl].lc_count : nr_if_none;
    o.nc = col_cl >= 0 ? cl[col_cl].lc_count : 1;
    o.cell_base = objs.empty() ? 0 : objs.back().cell_base + int64_t(objs.back().nr) * objs.back().nc;
    objs.push_back(o);  // its cells are made when a task first touches them (analyze)
    return int32_t(objs.size() - 1);
}

int32_t Planner::new_slot(int32_t init) {
    slot_init.push_back(init);
    return n_slots++;
}

int64_t Planner::plan_alloc(int64_t elems, int32_t temp_obj) {
    const int64_t off = *arena;
    *arena = align8(*arena + elems);
    plan_items.push_back(PlanItem{off, elems, temp_obj});
    return off;
}

// A temporary panel (rows x cols, column-major), its own region of the arena while the plan is
// emitted; relocate_temps later lets temporaries of the same shape and problem whose
// dependency-level intervals do not overlap share regions.
View Planner::new_temp(int32_t row_cl, int32_t rows, int32_t cols, int32_t rslot, int32_t cslot,
                       int32_t owner_cl) {
    View v;
    v.p.rows = rows;
    v.p.cols = cols;
    v.p.rslot = rslot;
    v.p.cslot = cslot;
    v.p.rs = 1;
    v.p.cs = rows;
    v.r_cl = row_cl;
    v.c_cl = -1;
    v.trans = false;
    v.obj = new_obj(row_cl, -1);
    const int64_t elems = int64_t(rows) * std::max(cols, 1);
    v.p.off = plan_alloc(elems, v.obj);
    note_temp(v.obj, elems, {owner_cl >= 0 && !inst.empty() ? inst[owner_cl] : -1, row_cl, rows, std::max(cols, 1)});
    return v;
}

// Registers object `obj` as a temporary of the current plan: its size and its shape (problem, row
// cluster, rows, columns; split-block factors carry their capacity as a negative column count, so
// that they share regions only with each other).
void Planner::note_temp(int32_t obj, int64_t elems, const std::array<int32_t, 4> &shape) {
    if ((int64_t)temp_size.size() <= obj) {  // the level intervals grow in analyze
        temp_size.resize(obj + 1, 0);
        temp_shape.resize(obj + 1, {-1, -1, -1, -1});
    }
    temp_size[obj] = elems;
    temp_shape[obj] = shape;
}

// Lets the product temporaries of plan p share regions: the plan's other allocations (split blocks,
// inverse blocks) are packed at the start of its range in their order, and the temporaries are laid
// out after them by their dependency-level intervals (first writer's level to last reader's): in
// order of first level, a temporary takes a free region of its exact size whose occupant's last
// level is below its first level, else a new one.  Every offset in the plan's descriptors (and in
// the stores and inverse blocks made during the plan) is moved accordingly, and for two temporaries
// that share a region every task that touches the earlier one becomes a predecessor of every task
// that writes the later one.  Those edges go from a lower level to a higher one, so the graph stays
// acyclic with the same levels (no longer dependency chain in levels).
int Planner::host_parts(int64_t limit) const {
    if (opt.batch_threads < 0) return 1;  // one thread (or one of a batch's pool of problem planners)
    const int64_t hw = std::max(1u, std::min(8u, std::thread::hardware_concurrency()));
    return int(std::max<int64_t>(1, std::min(hw, limit)));
}

void Planner::relocate_temps(Plan &p) {
    const size_t ni = plan_items.size();
    if (ni == 0) return;
    std::vector<int64_t> noff(ni, -1);
    int64_t pos = plan_begin;
    std::vector<size_t> tmp;
    for (size_t i = 0; i < ni; ++i) {
        if (plan_items[i].temp_obj < 0) {
            noff[i] = pos;
            pos = align8(pos + plan_items[i].size);
        } else {
            tmp.push_back(i);
        }
    }
    auto lev = [&](size_t i, bool last) {
        const int32_t o = plan_items[i].temp_obj;
        if (dep.temp_last[o] < 0) return 0;  // never touched
        return last ? dep.temp_last[o] : dep.temp_first[o];
    };
    {  // stable counting sort by first level (levels are below p.n_waves)
        std::vector<size_t> start(size_t(std::max(p.n_waves, 1)) + 1, 0), sorted(tmp.size());
        for (size_t i : tmp) start[lev(i, false) + 1]++;
        for (size_t k = 1; k < start.size(); ++k) start[k] += start[k - 1];
        for (size_t i : tmp) sorted[start[lev(i, false)]++] = i;
        tmp.swap(sorted);
    }
    // every temporary's shape (problem, row cluster, rows, cols) as a small integer
    struct ShapeHash {
        size_t operator()(const std::array<int32_t, 4> &a) const {
            uint64_t h = 0x9e3779b97f4a7c15ull;
            for (int32_t v : a) h = (h ^ uint32_t(v)) * 0xbf58476d1ce4e5b9ull;
            return size_t(h ^ (h >> 31));
        }
    };
    std::vector<int32_t> shape_of(ni, -1);
    int32_t n_shapes = 0;
    {
        std::unordered_map<std::array<int32_t, 4>, int32_t, ShapeHash> ids;
        ids.reserve(1024);
        for (size_t i : tmp) {
            auto it = ids.emplace(temp_shape[plan_items[i].temp_obj], n_shapes).first;
            if (it->second == n_shapes) ++n_shapes;
            shape_of[i] = it->second;
        }
    }
    // the temporaries placed so far by their last level; those of the levels below the current
    // temporary's first level are free again, released level by level and in item order
    std::vector<std::vector<int32_t>> ending(size_t(std::max(p.n_waves, 1)));
    int32_t released = 0;
    // free regions by shape: (offset, occupant)
    std::vector<std::vector<std::pair<int64_t, int32_t>>> free_by_shape(static_cast<size_t>(n_shapes));
    std::vector<std::pair<int32_t, int32_t>> order;  // (earlier temporary, later temporary) sharing a region
    int64_t top = pos;
    for (size_t i : tmp) {
        const int32_t f = lev(i, false);
        for (; released < f; ++released) {
            std::vector<int32_t> &done = ending[size_t(released)];
            std::sort(done.begin(), done.end());
            for (int32_t j : done) free_by_shape[shape_of[j]].emplace_back(noff[j], plan_items[j].temp_obj);
            std::vector<int32_t>().swap(done);
        }
        auto &fl = free_by_shape[shape_of[i]];
        if (!fl.empty()) {
            noff[i] = fl.back().first;
            order.emplace_back(fl.back().second, plan_items[i].temp_obj);
            fl.pop_back();
        } else {
            noff[i] = top;
            top = align8(top + plan_items[i].size);
        }
        ending[size_t(lev(i, true))].push_back(int32_t(i));
    }
    *arena = top;
    // the offsets in the plan move, and the shared regions add edges: the two on two threads
    auto remap_offsets = [&] {
        // offsets: an offset inside item k (items are in increasing offset order) keeps its distance.
        // The item of an offset is found from a table of the first item of every 4096-element page of
        // the plan's region, then a short forward scan (items are small: a few per page).
        constexpr int kPageShift = 12;
        const int64_t span = plan_items[ni - 1].off - plan_begin;
        std::vector<int32_t> page_item(size_t(span >> kPageShift) + 1);
        {
            size_t it = 0;
            for (size_t pg = 0; pg < page_item.size(); ++pg) {
                const int64_t start = plan_begin + (int64_t(pg) << kPageShift);
                while (it + 1 < ni && plan_items[it + 1].off <= start) ++it;
                page_item[pg] = int32_t(it);
            }
        }
        auto remap = [&](int64_t off) -> int64_t {
            if (off < plan_begin) return off;
            const size_t pg = std::min(size_t((off - plan_begin) >> kPageShift), page_item.size() - 1);
            size_t i = size_t(page_item[pg]);
            while (i + 1 < ni && plan_items[i + 1].off <= off) ++i;
            return noff[i] + (off - plan_items[i].off);
        };
        for (TGetrf &t : p.getrf) t.off = remap(t.off);
        for (TTrsm &t : p.trsm) {
            t.L_off = remap(t.L_off);
            t.P.off = remap(t.P.off);
        }
        for (TProject &t : p.project) {
            t.F.off = remap(t.F.off);
            t.X.off = remap(t.X.off);
            t.T.off = remap(t.T.off);
        }
        for (TAccum &t : p.accum) t.out.off = remap(t.out.off);
        for (Term &t : p.terms) {
            t.A.off = remap(t.A.off);
            t.X.off = remap(t.X.off);
        }
        for (TRadd &t : p.radd) {
            t.U_off = remap(t.U_off);
            t.V_off = remap(t.V_off);
        }
        for (Piece &t : p.pieces) {
            t.U.off = remap(t.U.off);
            t.V.off = remap(t.V.off);
        }
        for (TSplit &t : p.split) {
            t.srcU.off = remap(t.srcU.off);
            t.srcV.off = remap(t.srcV.off);
            t.dstU = remap(t.dstU);
            t.dstV = remap(t.dstV);
        }
        for (Store &st : fstore) {
            st.D_off = remap(st.D_off);
            st.U_off = remap(st.U_off);
            st.V_off = remap(st.V_off);
        }
        for (int64_t &o : inv_L_off) o = remap(o);
        for (int64_t &o : inv_U_off) o = remap(o);
    };
    auto add_edges = [&] {
        if (order.empty()) return;
        // the touches of every temporary (counting sort by object; a task's touches are in cell order)
        const size_t nobj = temp_size.size();
        std::vector<int32_t> tptr(nobj + 1, 0), ttask(dep.touch_obj.size()), tcell(dep.touch_obj.size());
        std::vector<uint8_t> twr(dep.touch_obj.size());
        for (int32_t o : dep.touch_obj) tptr[o + 1]++;
        for (size_t o = 0; o < nobj; ++o) tptr[o + 1] += tptr[o];
        {
            std::vector<int32_t> fill(tptr.begin(), tptr.end() - 1);
            for (size_t e = 0; e < dep.touch_obj.size(); ++e) {
                const int32_t at = fill[dep.touch_obj[e]]++;
                ttask[at] = dep.touch_task[e];
                tcell[at] = dep.touch_cell[e];
                twr[at] = dep.touch_write[e];
            }
        }
        // per shared region, cell by cell (the two temporaries have the same shape, hence the same
        // cells): every task that touched the earlier one's cell precedes every writer of the later one's
        // (split by ranges of region pairs over host threads, put side by side in pair order)
        const int npairs = host_parts(int64_t(order.size()) / 16384 + 1);
        std::vector<std::vector<std::pair<int32_t, int32_t>>> part_extra(static_cast<size_t>(npairs));
        run_parts(npairs, [&](int q) {
            std::vector<std::pair<int32_t, int32_t>> &extra = part_extra[size_t(q)];  // (task, predecessor)
            std::vector<std::vector<int32_t>> by_cell;
            const size_t k0 = order.size() * size_t(q) / size_t(npairs);
            const size_t k1 = order.size() * size_t(q + 1) / size_t(npairs);
            for (size_t k = k0; k < k1; ++k) {
                const int32_t a = order[k].first, b = order[k].second;
                const int32_t ncell = objs[a].nr * objs[a].nc;
                if ((int32_t)by_cell.size() < ncell) by_cell.resize(ncell);
                for (int32_t c = 0; c < ncell; ++c) by_cell[c].clear();
                for (int32_t e = tptr[a]; e < tptr[a + 1]; ++e) by_cell[tcell[e]].push_back(ttask[e]);
                for (int32_t e = tptr[b]; e < tptr[b + 1]; ++e)
                    if (twr[e])
                        for (int32_t t : by_cell[tcell[e]]) extra.emplace_back(ttask[e], t);
            }
        });
        std::vector<std::pair<int32_t, int32_t>> extra;
        {
            size_t total = 0;
            for (const auto &v : part_extra) total += v.size();
            extra.reserve(total);
            for (auto &v : part_extra) {
                extra.insert(extra.end(), v.begin(), v.end());
                std::vector<std::pair<int32_t, int32_t>>().swap(v);
            }
        }
        // merge into the predecessor lists (CSR), each predecessor once per task (the extra edges
        // grouped by task with a counting sort)
        const int64_t nt = p.n_tasks;
        std::vector<int32_t> xptr(nt + 1, 0), xidx(extra.size());
        for (const auto &e : extra) xptr[e.first + 1]++;
        for (int64_t g = 0; g < nt; ++g) xptr[g + 1] += xptr[g];
        {
            std::vector<int32_t> fill(xptr.begin(), xptr.end() - 1);
            for (const auto &e : extra) xidx[fill[e.first]++] = e.second;
        }
        // the merge of a task depends on its own lists only: split by task ranges over host threads,
        // each part merging into its own list, then the parts put side by side
        const int nparts = host_parts(nt / 65536 + 1);
        std::vector<std::vector<int32_t>> part_idx(static_cast<size_t>(nparts));
        std::vector<int32_t> nptr(nt + 1, 0);  // first the merged length of every task
        run_parts(nparts, [&](int q) {
            const int64_t g0 = nt * q / nparts, g1 = nt * (q + 1) / nparts;
            std::vector<int32_t> &out = part_idx[size_t(q)];
            out.reserve(size_t(p.pred_ptr[g1] - p.pred_ptr[g0]) + size_t(xptr[g1] - xptr[g0]));
            std::vector<int32_t> mark(nt, -1);
            for (int64_t g = g0; g < g1; ++g) {
                const size_t before = out.size();
                if (xptr[g] == xptr[g + 1]) {  // no extra edge: the list as it is (already without repeats)
                    out.insert(out.end(), p.pred_idx.begin() + p.pred_ptr[g], p.pred_idx.begin() + p.pred_ptr[g + 1]);
                } else {
                    for (int32_t e = p.pred_ptr[g]; e < p.pred_ptr[g + 1]; ++e) {
                        const int32_t t = p.pred_idx[e];
                        if (mark[t] != g) {
                            mark[t] = int32_t(g);
                            out.push_back(t);
                        }
                    }
                    for (int32_t e = xptr[g]; e < xptr[g + 1]; ++e) {
                        const int32_t t = xidx[e];
                        if (t != g && mark[t] != g) {
                            mark[t] = int32_t(g);
                            out.push_back(t);
                        }
                    }
                }
                nptr[g + 1] = int32_t(out.size() - before);
            }
        });
        for (int64_t g = 0; g < nt; ++g) nptr[g + 1] += nptr[g];
        std::vector<int32_t> nidx(static_cast<size_t>(nptr[nt]));
        run_parts(nparts, [&](int q) {
            const int64_t g0 = nt * q / nparts;
            std::copy(part_idx[size_t(q)].begin(), part_idx[size_t(q)].end(), nidx.begin() + nptr[g0]);
            std::vector<int32_t>().swap(part_idx[size_t(q)]);
        });
        p.pred_ptr.swap(nptr);
        p.pred_idx.swap(nidx);
    };
    const int two = host_parts(2);
    run_parts(two, [&](int q) {
        if (q == 0) add_edges();
        if (q == 1 || two == 1) remap_offsets();
    });
}

// The largest sum of temporary elements in use at one dependency level (the memory an allocation
// of regions by non-overlapping level intervals would need; a lower bound for any that adds no level).
void Planner::temp_levels(Plan &p) const {
    std::vector<int64_t> delta(size_t(p.n_waves) + 2, 0);
    int64_t tot = 0;
    for (size_t o = 0; o < temp_size.size(); ++o) {
        if (temp_size[o] == 0 || dep.temp_last[o] < 0) continue;
        tot += temp_size[o];
        delta[dep.temp_first[o]] += temp_size[o];
        delta[dep.temp_last[o] + 1] -= temp_size[o];
    }
    int64_t cur = 0, peak = 0;
    for (int64_t d : delta) {
        cur += d;
        peak = std::max(peak, cur);
    }
    p.temp_elems = tot;
    p.temp_peak_elems = peak;
}


void Planner::describe(const View &v, ViewRec &r) const {
    const Obj &o = objs[v.obj];
    const int32_t vr = v.trans ? v.c_cl : v.r_cl;  // cluster restricting object rows
    const int32_t vc = v.trans ? v.r_cl : v.c_cl;  // cluster restricting object columns
    r.base = o.cell_base;
    r.nc = o.nc;
    r.r0 = 0;
    r.r1 = o.nr;
    r.c0 = 0;
    r.c1 = o.nc;
    if (o.row_cl >= 0 && vr >= 0) {
        r.r0 = cl[vr].lc_first - cl[o.row_cl].lc_first;
        r.r1 = r.r0 + cl[vr].lc_count;
    }
    if (o.col_cl >= 0 && vc >= 0) {
        r.c0 = cl[vc].lc_first - cl[o.col_cl].lc_first;
        r.c1 = r.c0 + cl[vc].lc_count;
    }
    r.temp_obj = v.obj < (int32_t)temp_size.size() && temp_size[v.obj] > 0 ? v.obj : -1;
}

void Planner::cells_of(const View &v, std::vector<int64_t> &out) const {
    ViewRec r;
    describe(v, r);
    for (int32_t a = r.r0; a < r.r1; ++a)
        for (int32_t c = r.c0; c < r.c1; ++c) out.push_back(r.base + int64_t(a) * r.nc + c);
}

int32_t Planner::analyze(Deps &d, std::vector<int32_t> &pred_ptr, std::vector<int32_t> &pred_idx, const ViewRec *v,
                         size_t nr, size_t nw, int32_t g) const {
    static thread_local std::vector<int64_t> rc, wc;
    static thread_local std::vector<size_t> rend, wend;  // end of every view's cells in rc / wc
    rc.clear();
    wc.clear();
    rend.clear();
    wend.clear();
    for (size_t i = 0; i < nr + nw; ++i) {
        const ViewRec &r = v[i];
        std::vector<int64_t> &out = i < nr ? rc : wc;
        if (r.r1 > r.r0 && r.c1 > r.c0) {
            const int64_t end = r.base + int64_t(r.r1 - 1) * r.nc + r.c1;  // cells are made on first use
            if ((int64_t)d.cell.size() < end) d.cell.resize(end, CellState{-1, -1, -1, -1});
            for (int32_t a = r.r0; a < r.r1; ++a)
                for (int32_t c = r.c0; c < r.c1; ++c) out.push_back(r.base + int64_t(a) * r.nc + c);
        }
        (i < nr ? rend : wend).push_back(out.size());
    }
    int32_t dep = -1;
    for (int64_t c : rc) dep = std::max(dep, d.cell[c].write_wave);
    for (int64_t c : wc) dep = std::max(dep, std::max(d.cell[c].write_wave, d.cell[c].read_wave));
    const int32_t w = dep + 1;
    for (size_t i = 0; i < nr + nw; ++i) {  // the level interval and the cells of the temporaries touched
        const int32_t o = v[i].temp_obj;
        if (o < 0) continue;
        if ((int32_t)d.temp_first.size() <= o) {
            d.temp_first.resize(size_t(o) + 1, INT32_MAX);
            d.temp_last.resize(size_t(o) + 1, -1);
        }
        d.temp_first[o] = std::min(d.temp_first[o], w);
        d.temp_last[o] = std::max(d.temp_last[o], w);
        if (!opt.temp_reuse) continue;  // the cell touches only order shared regions
        const bool wr = i >= nr;
        const std::vector<int64_t> &cv = wr ? wc : rc;
        const size_t j = wr ? i - nr : i;
        const size_t b = j ? (wr ? wend : rend)[j - 1] : 0, e = (wr ? wend : rend)[j];
        for (size_t k = b; k < e; ++k) {
            d.touch_obj.push_back(o);
            d.touch_cell.push_back(int32_t(cv[k] - v[i].base));
            d.touch_task.push_back(g);
            d.touch_write.push_back(wr ? 1 : 0);
        }
    }
    for (int64_t c : rc) d.cell[c].read_wave = std::max(d.cell[c].read_wave, w);
    for (int64_t c : wc) {
        d.cell[c].write_wave = w;
        d.cell[c].read_wave = -1;
    }
    // explicit edges: read-after-write, write-after-write, write-after-read; each predecessor is
    // listed once (d.pred_mark[t] == g once t is in this task's list), in the order first met
    if (pred_ptr.empty()) pred_ptr.push_back(0);
    if ((int64_t)d.pred_mark.size() < (int64_t)g + 1) d.pred_mark.resize(std::max<int64_t>(2 * (int64_t)g, 1024), -1);
    auto add = [&](int32_t t) {
        if (t >= 0 && t != g && d.pred_mark[t] != g) {
            d.pred_mark[t] = g;
            pred_idx.push_back(t);
        }
    };
    for (int64_t c : rc) add(d.cell[c].writer);
    for (int64_t c : wc) {
        add(d.cell[c].writer);
        for (int32_t e = d.cell[c].rhead; e >= 0; e = d.rpool_next[e]) add(d.rpool_task[e]);
    }
    pred_ptr.push_back(int32_t(pred_idx.size()));
    for (int64_t c : rc) {
        d.rpool_task.push_back(g);
        d.rpool_next.push_back(d.cell[c].rhead);
        d.cell[c].rhead = int32_t(d.rpool_task.size() - 1);
    }
    for (int64_t c : wc) {
        d.cell[c].writer = g;
        d.cell[c].rhead = -1;
    }
    return w;
}

// The hand-over between emission and analysis: a ring of chunks of task records (the number of
// read and written views, then their cell rectangles), filled by the emitting thread and taken in
// order by the analysing thread, which owns the cell states, the predecessor lists, the level
// intervals of the temporaries and the waves until pipe_end.
struct Planner::Pipe {
    static constexpr size_t kRing = 4, kTasks = 2048;
    struct Chunk {
        std::vector<uint32_t> counts;  // per task: its reads, then its writes
        std::vector<ViewRec> views;
    };
    Chunk ring[kRing];
    alignas(64) size_t produced = 0, consumed = 0;  // chunks handed over / analysed
    bool done = false, failed = false;
    std::mutex mu;
    std::condition_variable cv;
    std::thread th;
    // the analysing thread's own (cache lines apart from what the emitting thread writes)
    alignas(64) Deps d;
    std::vector<int32_t> pred_ptr, pred_idx;
    std::vector<int32_t> waves;  // per task from task g0 on
    int32_t g0 = 0, n_waves = 0;
    alignas(64) char pad_ = 0;  // keeps the fields above off the cache line of what follows

    Chunk &current() { return ring[produced % kRing]; }
    // hands the current chunk over and waits until the next one in the ring has been analysed
    void publish() {
        std::unique_lock<std::mutex> lk(mu);
        ++produced;
        cv.notify_all();
        cv.wait(lk, [&] { return produced - consumed < kRing; });
        Chunk &c = current();
        c.counts.clear();
        c.views.clear();
    }
};

bool Planner::pipe_begin() {
    pipe = new Pipe();
    Pipe *q = pipe;
    q->d.swap(dep);
    q->pred_ptr.swap(P->pred_ptr);
    q->pred_idx.swap(P->pred_idx);
    q->g0 = int32_t(P->n_tasks);
    auto work = [this, q] {
        int32_t g = q->g0;
        for (;;) {
            size_t idx;
            {
                std::unique_lock<std::mutex> lk(q->mu);
                q->cv.wait(lk, [&] { return q->consumed < q->produced || q->done; });
                if (q->consumed == q->produced) return;
                idx = q->consumed % Pipe::kRing;
            }
            const Pipe::Chunk &c = q->ring[idx];
            if (!q->failed) {
                try {
                    size_t at = 0;
                    for (size_t t = 0; t < c.counts.size(); t += 2) {
                        const size_t nr = c.counts[t], nw = c.counts[t + 1];
                        const int32_t w = analyze(q->d, q->pred_ptr, q->pred_idx, c.views.data() + at, nr, nw, g++);
                        q->waves.push_back(w);
                        q->n_waves = std::max(q->n_waves, w + 1);
                        at += nr + nw;
                    }
                } catch (const std::bad_alloc &) {
                    q->failed = true;
                }
            }
            std::lock_guard<std::mutex> lk(q->mu);
            ++q->consumed;
            q->cv.notify_all();
        }
    };
    try {
        q->th = std::thread(work);
    } catch (const std::system_error &) {  // no thread to be had: the analysis stays on this one
        dep.swap(q->d);
        P->pred_ptr.swap(q->pred_ptr);
        P->pred_idx.swap(q->pred_idx);
        delete q;
        pipe = nullptr;
        return false;
    }
    return true;
}

int Planner::pipe_end() {
    Pipe *q = pipe;
    pipe = nullptr;
    {
        std::lock_guard<std::mutex> lk(q->mu);
        if (!q->current().counts.empty()) ++q->produced;  // the last, partial chunk
        q->done = true;
        q->cv.notify_all();
    }
    q->th.join();
    dep.swap(q->d);
    P->pred_ptr.swap(q->pred_ptr);
    P->pred_idx.swap(q->pred_idx);
    const bool failed = q->failed;
    if (!failed) {  // the waves into the kinds' lists, in emission order
        for (size_t i = 0; i < q->waves.size(); ++i) {
            const int32_t code = P->task_code[size_t(q->g0) + i];
            P->wave[code >> kCodeShift][code & kCodeMask] = q->waves[i];
        }
        P->n_waves = std::max(P->n_waves, q->n_waves);
    }
    delete q;
    if (failed) {
        error = "out of host memory in the dependency analysis";
        return HLU_ENOMEM;
    }
    return HLU_OK;
}

int32_t Planner::emit_views(Kind k, const View *const *reads, size_t nr, const View *const *writes, size_t nw) {
    static thread_local std::vector<ViewRec> local;
    ViewRec *v;
    if (pipe) {
        std::vector<ViewRec> &dst = pipe->current().views;
        dst.resize(dst.size() + nr + nw);
        v = dst.data() + dst.size() - (nr + nw);
    } else {
        local.resize(nr + nw);
        v = local.data();
    }
    for (size_t i = 0; i < nr; ++i) describe(*reads[i], v[i]);
    for (size_t i = 0; i < nw; ++i) describe(*writes[i], v[nr + i]);
    int32_t w = 0;
    if (pipe) {
        Pipe::Chunk &c = pipe->current();
        c.counts.push_back(uint32_t(nr));
        c.counts.push_back(uint32_t(nw));
        if (c.counts.size() >= 2 * Pipe::kTasks) pipe->publish();
    } else {
        w = analyze(dep, P->pred_ptr, P->pred_idx, v, nr, nw, int32_t(P->n_tasks));
        P->n_waves = std::max(P->n_waves, w + 1);
    }
    P->task_code.push_back((int32_t(k) << kCodeShift) | int32_t(P->wave[k].size()));
    P->wave[k].push_back(w);  // the analysing thread's wave is filled in by pipe_end
    P->n_tasks++;
    return w;
}

// -------------------------------------------------------------------- views
View Planner::viewD(const Block *b) {
    Store &s = st(b);
    View v;
    v.p = Panel{s.D_off, s.m, s.n, -1, -1, 1, s.m};
    v.obj = s.objD;
    v.r_cl = b->t;
    v.c_cl = b->s;
    v.trans = false;
    return v;
}

View Planner::viewU(const Block *b) {
    Store &s = st(b);
    View v;
    v.p = Panel{s.U_off, s.m, s.kslot >= 0 ? s.cap : s.krank, -1, s.kslot, 1, s.m};
    v.obj = s.objU;
    v.r_cl = b->t;
    v.c_cl = -1;
    v.trans = false;
    return v;
}

View Planner::viewV(const Block *b) {
    Store &s = st(b);
    View v;
    v.p = Panel{s.V_off, s.n, s.kslot >= 0 ? s.cap : s.krank, -1, s.kslot, 1, s.n};
    v.obj = s.objV;
    v.r_cl = b->s;
    v.c_cl = -1;
    v.trans = false;
    return v;
}

View Planner::ident(int32_t c) {
    View v;
    v.p = Panel{f_ident_off, cl[c].size, cl[c].size, -1, -1, 1, max_leaf};
    v.obj = ident_obj;
    v.r_cl = c;
    v.c_cl = c;
    v.trans = false;
    return v;
}

View Planner::rows(const View &v, int32_t sub) const {
    View r = v;
    int64_t d = int64_t(cl[sub].begin) - cl[v.r_cl].begin;
    r.p.off += d * v.p.rs;
    r.p.rows = cl[sub].size;
    r.p.rslot = -1;
    r.r_cl = sub;
    return r;
}

View Planner::transpose(const View &v) {
    View t = v;
    std::swap(t.p.rows, t.p.cols);
    std::swap(t.p.rslot, t.p.cslot);
    std::swap(t.p.rs, t.p.cs);
    std::swap(t.r_cl, t.c_cl);
    t.trans = !v.trans;
    return t;
}

void Planner::collect_leaves(Block *b, std::vector<Block *> &out) {
    if (b->kind == B_ZERO) return;
    if (b->kind == B_PART) {
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) collect_leaves(b->son[i][j], out);
    } else {
        out.push_back(b);
    }
}

// ----------------------------------------------------- the H-LU recursion
// lu: the 2 x 2 block LU recursion of Sec. 3.1 at a partitioned diagonal block (factor the leading
// block, solve both off-diagonal panels with its factors, Schur update, factor the trailing block),
// getrf at a dense leaf.
void Planner::lu(Block *b) {
    if (b->kind == B_DENSE) {
        Store &s = st(b);
        View D = viewD(b);
        P->getrf.push_back(TGetrf{s.D_off, s.m, b->id});
        emit(K_GETRF, {}, {&D});
        return;
    }
    lu(b->son[0][0]);
    trsm_l(b->son[0][0], b->son[0][1]);
    trsm_u(b->son[0][0], b->son[1][0]);
    addmul(b->son[1][1], -1.0, b->son[1][0], b->son[0][1]);
    lu(b->son[1][1]);
}

void Planner::trsm_l(Block *L, Block *X) {
    if (X->kind == B_ZERO) return;
    if (X->kind == B_LOWRANK) {
        trsm_l_panel(L, viewU(X));  // L^{-1} U V^T: solve on the k columns of U
    } else if (X->kind == B_DENSE) {
        trsm_l_panel(L, viewD(X));
    } else {  // block substitution: first block row, Schur update, second block row
        for (int j = 0; j < 2; ++j) trsm_l(L->son[0][0], X->son[0][j]);
        for (int j = 0; j < 2; ++j) addmul(X->son[1][j], -1.0, L->son[1][0], X->son[0][j]);
        for (int j = 0; j < 2; ++j) trsm_l(L->son[1][1], X->son[1][j]);
    }
}

void Planner::trsm_u(Block *U, Block *X) {
    if (X->kind == B_ZERO) return;
    if (X->kind == B_LOWRANK) {
        trsm_u_panel(U, viewV(X));  // U V^T R^{-1} = U (R^{-T} V)^T: solve on the rows of V
    } else if (X->kind == B_DENSE) {
        trsm_u_panel(U, transpose(viewD(X)));  // X R^{-1} = (R^{-T} X^T)^T
    } else {
        for (int i = 0; i < 2; ++i) trsm_u(U->son[0][0], X->son[i][0]);
        for (int i = 0; i < 2; ++i) addmul(X->son[i][1], -1.0, X->son[i][0], U->son[0][1]);
        for (int i = 0; i < 2; ++i) trsm_u(U->son[1][1], X->son[i][1]);
    }
}

void Planner::trsm_l_panel(Block *L, const View &Pv) {
    if (L->kind == B_DENSE) {
        Store &s = st(L);
        View D = viewD(L);
        P->trsm.push_back(TTrsm{s.D_off, s.m, TR_LOWER_UNIT, Pv.p});
        emit(K_TRSM, {&D}, {&Pv});
        return;
    }
    int32_t t0 = cl[L->t].son0, t1 = cl[L->t].son1;
    trsm_l_panel(L->son[0][0], rows(Pv, t0));
    hmm(rows(Pv, t1), -1.0, false, L->son[1][0], false, rows(Pv, t0));
    trsm_l_panel(L->son[1][1], rows(Pv, t1));
}

// P := R^{-T} P with R the upper factor of U's diagonal block (rows of P = U->t)
void Planner::trsm_u_panel(Block *U, const View &Pv) {
    if (U->kind == B_DENSE) {
        Store &s = st(U);
        View D = viewD(U);
        P->trsm.push_back(TTrsm{s.D_off, s.m, TR_UPPER_TRANS, Pv.p});
        emit(K_TRSM, {&D}, {&Pv});
        return;
    }
    int32_t t0 = cl[U->t].son0, t1 = cl[U->t].son1;
    trsm_u_panel(U->son[0][0], rows(Pv, t0));
    hmm(rows(Pv, t1), -1.0, false, U->son[0][1], true, rows(Pv, t0));
    trsm_u_panel(U->son[1][1], rows(Pv, t1));
}

// out (+)= alpha * op(M) X, op(M) = M or M^T, exact (Sec. 3.1: U (V^T X) on
// low-rank leaves).  Phase 1 projects every low-rank leaf, phase 2 sums the
// contributions of all leaves covering one leaf cluster of the output rows.
void Planner::hmm(const View &out, double alpha, bool overwrite, Block *M, bool trans, const View &X,
                  int32_t wdst, int32_t wsrc) {
    // scratch reused across calls (hmm does not recurse)
    static thread_local std::vector<Block *> lv;
    static thread_local std::vector<View> Tv;
    static thread_local std::vector<std::vector<int32_t>> seg;
    static thread_local std::vector<View> keep;
    static thread_local std::vector<const View *> rd;
    static thread_local std::vector<int32_t> depth, group;
    static thread_local std::vector<int64_t> cells;
    lv.clear();
    collect_leaves(M, lv);
    Tv.assign(lv.size(), View{});
    for (size_t i = 0; i < lv.size(); ++i) {
        Block *m = lv[i];
        if (m->kind != B_LOWRANK) continue;
        Store &s = st(m);
        View F = trans ? viewU(m) : viewV(m);
        View Xs = rows(X, trans ? m->t : m->s);
        int32_t krows = F.p.cslot >= 0 ? s.cap : F.p.cols;
        View T = new_temp(-1, krows, X.p.cols, F.p.cslot, X.p.cslot, m->t);
        TProject tp{F.p, Xs.p, T.p, -1, -1, -1, -1, no_flops ? 1 : 0, 0};
        P->project.push_back(tp);
        emit(K_PROJECT, {&F, &Xs}, {&T});
        Tv[i] = T;
    }
    int32_t oc = out.r_cl;
    int32_t lc0 = cl[oc].lc_first, nseg = cl[oc].lc_count;
    if ((int32_t)seg.size() < nseg) seg.resize(nseg);
    for (int32_t qi = 0; qi < nseg; ++qi) seg[qi].clear();
    for (size_t i = 0; i < lv.size(); ++i) {
        int32_t rm = trans ? lv[i]->s : lv[i]->t;
        for (int32_t q = cl[rm].lc_first; q < cl[rm].lc_first + cl[rm].lc_count; ++q)
            seg[q - lc0].push_back(int32_t(i));
    }
    for (int32_t qi = 0; qi < nseg; ++qi) {
        if (seg[qi].empty() && !overwrite) continue;
        int32_t q = lc_ids[lc0 + qi];
        View o = rows(out, q);
        const size_t nt = seg[qi].size();
        keep.assign(2 * nt, View{});
        depth.assign(nt, -1);
        for (size_t ti = 0; ti < nt; ++ti) {
            Block *m = lv[seg[qi][ti]];
            if (m->kind == B_DENSE) {
                keep[2 * ti] = rows(trans ? transpose(viewD(m)) : viewD(m), q);
                keep[2 * ti + 1] = rows(X, trans ? m->t : m->s);
            } else {
                keep[2 * ti] = rows(trans ? viewV(m) : viewU(m), q);
                keep[2 * ti + 1] = Tv[seg[qi][ti]];
            }
            // depth of the term (solve plan only): the latest dependency level among the cells it reads
            if (split_accum) {
                cells.clear();
                cells_of(keep[2 * ti], cells);
                cells_of(keep[2 * ti + 1], cells);
                for (int64_t c : cells)
                    if (c < (int64_t)dep.cell.size()) depth[ti] = std::max(depth[ti], dep.cell[c].write_wave);
            }
        }
        // In the solve, the terms whose inputs are ready at the deepest level (the part of the
        // update that waits on the latest solved segment) get their own ACCUM; the others are
        // summed first, off that path.  Both sums go into the same output in the same order
        // of terms within each group.
        group.clear();
        const int32_t dmax = nt ? *std::max_element(depth.begin(), depth.end()) : -1;
        bool split = false;
        if (split_accum && nt > 1)
            for (size_t ti = 0; ti < nt; ++ti) split = split || depth[ti] < dmax;
        for (int pass = 0; pass < (split ? 2 : 1); ++pass) {
            const bool late = split && pass == 1;
            const bool first = pass == 0;
            int32_t cnt = 0;
            const int32_t t0 = int32_t(P->terms.size());
            rd.clear();
            for (size_t ti = 0; ti < nt; ++ti) {
                if (split && ((depth[ti] == dmax) != late)) continue;
                P->terms.push_back(Term{keep[2 * ti].p, keep[2 * ti + 1].p});
                rd.push_back(&keep[2 * ti]);
                rd.push_back(&keep[2 * ti + 1]);
                ++cnt;
            }
            const bool ow = overwrite && first;
            P->accum.push_back(TAccum{o.p, alpha, ow ? 1 : 0, t0, cnt, wdst, wsrc, no_flops ? -1.0f : 0.0f});
            if (!ow) rd.push_back(&o);
            emit(K_ACCUM, rd, {&o});
        }
    }
}

Planner::Prod Planner::product(Block *A, Block *B) {
    if (A->kind == B_LOWRANK) {  // (U_a V_a^T) B = U_a (B^T V_a)^T
        Store &sa = st(A);
        int32_t ws = new_slot(0);
        View W = new_temp(B->s, cl[B->s].size, sa.cap, -1, ws, B->s);
        hmm(W, 1.0, true, B, true, viewV(A), ws, sa.kslot);
        return Prod{viewU(A), W};
    }
    if (B->kind == B_LOWRANK) {  // A (U_b V_b^T) = (A U_b) V_b^T
        Store &sb = st(B);
        int32_t ws = new_slot(0);
        View W = new_temp(A->t, cl[A->t].size, sb.cap, -1, ws, A->t);
        hmm(W, 1.0, true, A, false, viewU(B), ws, sb.kslot);
        return Prod{W, viewV(B)};
    }
    int32_t tsz = cl[A->t].size, rsz = cl[A->s].size, ssz = cl[B->s].size;
    if (A->kind == B_DENSE && B->kind == B_DENSE && rsz <= std::min(tsz, ssz))
        return Prod{viewD(A), transpose(viewD(B))};  // factors of the product itself
    if (A->kind == B_DENSE && (B->kind == B_PART || tsz <= ssz)) {
        // A B = I_t (B^T A^T)^T with the leaf cluster t on the identity side
        View W = new_temp(B->s, ssz, tsz, -1, -1, B->s);
        hmm(W, 1.0, true, B, true, transpose(viewD(A)));
        return Prod{ident(A->t), W};
    }
    // A B = (A D_B) I_s^T with the leaf cluster s on the identity side
    View W = new_temp(A->t, tsz, ssz, -1, -1, A->t);
    hmm(W, 1.0, true, A, false, viewD(B));
    return Prod{W, ident(B->s)};
}

void Planner::add_into(Block *C, double alpha, const Prod &p) {
    if (C->kind == B_PART) {
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) {
                Block *c = C->son[i][j];
                add_into(c, alpha, Prod{rows(p.U, c->t), rows(p.V, c->s)});
            }
        return;
    }
    if (C->kind == B_DENSE) {
        View D = viewD(C);
        View Vt = transpose(p.V);
        for (int32_t qi = 0; qi < cl[C->t].lc_count; ++qi) {
            int32_t q = lc_ids[cl[C->t].lc_first + qi];
            View o = rows(D, q);
            View A = rows(p.U, q);
            P->accum.push_back(TAccum{o.p, alpha, 0, int32_t(P->terms.size()), 1, -1, -1, 0.0f});
            P->terms.push_back(Term{A.p, Vt.p});
            emit(K_ACCUM, {&A, &Vt, &o}, {&o});
        }
        return;
    }
    Piece pc{alpha, p.U.p, p.V.p, 0, 0};
    radd(C, true, {pc}, {p.U, p.V});
}

void Planner::radd(Block *C, bool include_self, const std::vector<Piece> &pcs,
                   const std::vector<View> &pviews) {
    Store &s = st(C);
    int32_t kcap = include_self ? s.cap : 0;
    for (const Piece &pc : pcs) kcap += pc.U.cols;
    TRadd tr{};
    tr.U_off = s.U_off;
    tr.V_off = s.V_off;
    tr.scratch_off = 0;
    tr.m = s.m;
    tr.n = s.n;
    tr.cap = s.cap;
    tr.kslot = s.kslot;
    tr.include_self = include_self ? 1 : 0;
    tr.piece0 = int32_t(P->pieces.size());
    tr.npieces = int32_t(pcs.size());
    tr.Kcap = kcap;
    tr.target = C->id;
    tr.inst = inst.empty() ? 0 : std::max(0, inst[C->t]);
    for (const Piece &pc : pcs) P->pieces.push_back(pc);
    P->radd.push_back(tr);
    P->max_kcap = std::max(P->max_kcap, kcap);
    View U = viewU(C), V = viewV(C);
    static thread_local std::vector<const View *> rd;
    rd.clear();
    for (const View &v : pviews) rd.push_back(&v);
    if (include_self) {
        rd.push_back(&U);
        rd.push_back(&V);
    }
    emit(K_RADD, rd, {&U, &V});
}

void Planner::addmul(Block *C, double alpha, Block *A, Block *B) {
    if (C->kind == B_ZERO || A->kind == B_ZERO || B->kind == B_ZERO) return;  // no coupling between instances
    if (A->kind == B_PART && B->kind == B_PART) {
        if (C->kind == B_PART) {
            for (int i = 0; i < 2; ++i)
                for (int j = 0; j < 2; ++j)
                    for (int k = 0; k < 2; ++k) addmul(C->son[i][j], alpha, A->son[i][k], B->son[k][j]);
            return;
        }
        // low-rank target, both factors partitioned: temporary 2x2 split
        Store cs = st(C);
        Block *S[2][2];
        View CU = viewU(C), CV = viewV(C);
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) {
                int32_t ti = A->son[i][0]->t, sj = B->son[0][j]->s;
                Block *v = new Block{ti, sj, B_LOWRANK, int32_t(fstore.size()), {{nullptr, nullptr}, {nullptr, nullptr}}};
                blocks_owned.push_back(v);
                Store vs{};
                vs.kind = B_LOWRANK;
                vs.t = ti;
                vs.s = sj;
                vs.m = cl[ti].size;
                vs.n = cl[sj].size;
                vs.cap = std::max(std::min(std::min(vs.m, vs.n), opt.rank_cap), cs.cap);
                vs.kslot = new_slot(0);
                vs.krank = 0;
                vs.objU = new_obj(ti, -1);
                vs.objV = new_obj(sj, -1);
                // the son's factors live from the split to the merge: temporaries of the plan
                vs.U_off = plan_alloc(int64_t(vs.m) * vs.cap, vs.objU);
                vs.V_off = plan_alloc(int64_t(vs.n) * vs.cap, vs.objV);
                note_temp(vs.objU, int64_t(vs.m) * vs.cap, {ti >= 0 && !inst.empty() ? inst[ti] : -1, ti, vs.m, -vs.cap});
                note_temp(vs.objV, int64_t(vs.n) * vs.cap, {sj >= 0 && !inst.empty() ? inst[sj] : -1, sj, vs.n, -vs.cap});
                vs.objD = -1;
                fstore.push_back(vs);
                S[i][j] = v;
                View su = rows(CU, ti), sv = rows(CV, sj);
                View du = viewU(v), dv = viewV(v);
                P->split.push_back(TSplit{su.p, sv.p, vs.U_off, vs.V_off, vs.m, vs.n, cs.kslot, vs.kslot});
                emit(K_SPLIT, {&su, &sv}, {&du, &dv});
            }
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j)
                for (int k = 0; k < 2; ++k) addmul(S[i][j], alpha, A->son[i][k], B->son[k][j]);
        std::vector<Piece> pcs;
        std::vector<View> pv;
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) {
                View u = viewU(S[i][j]), v = viewV(S[i][j]);
                pcs.push_back(Piece{1.0, u.p, v.p, cl[S[i][j]->t].begin - cl[C->t].begin,
                                    cl[S[i][j]->s].begin - cl[C->s].begin});
                pv.push_back(u);
                pv.push_back(v);
            }
        radd(C, false, pcs, pv);
        return;
    }
    Prod p = product(A, B);
    add_into(C, alpha, p);
}

// --------------------------------------------------------------- the solve
void Planner::solve_lower(Block *F, const View &Y) {
    if (F->kind == B_DENSE) {
        Store &s = st(F);
        View D = viewD(F);
        P->trsm.push_back(TTrsm{s.D_off, s.m, TR_LOWER_UNIT, Y.p});
        emit(K_TRSM, {&D}, {&Y});
        return;
    }
    int32_t t0 = cl[F->t].son0, t1 = cl[F->t].son1;
    solve_lower(F->son[0][0], rows(Y, t0));
    hmm(rows(Y, t1), -1.0, false, F->son[1][0], false, rows(Y, t0));
    solve_lower(F->son[1][1], rows(Y, t1));
}

void Planner::solve_upper(Block *F, const View &Y) {
    if (F->kind == B_DENSE) {
        Store &s = st(F);
        View D = viewD(F);
        P->trsm.push_back(TTrsm{s.D_off, s.m, TR_UPPER, Y.p});
        emit(K_TRSM, {&D}, {&Y});
        return;
    }
    int32_t t0 = cl[F->t].son0, t1 = cl[F->t].son1;
    solve_upper(F->son[1][1], rows(Y, t1));
    hmm(rows(Y, t0), -1.0, false, F->son[0][1], false, rows(Y, t1));
    solve_upper(F->son[0][0], rows(Y, t0));
}

// ------------------------------------------------------ inverse-block solve
// The block forward substitution of Sec. 3.1 (solve(F00); y1 -= F10 x0; solve(F11)) is kept above
// a chosen level of diagonal blocks (c, c); below it, x_c = L_cc^{-1} y_c and x_c = U_cc^{-1} z_c are
// applied as dense products.  The inverses are formed at the end of the factorisation by the same
// substitution applied to the identity, one leaf cluster of columns at a time (n_c / leaf
// independent chains per block, all off the factorisation's own path).  The solve's chain then has
// one product per inverse block instead of one triangular solve and one update per leaf cluster.

// Whether the block-tree leaf that covers rows of cluster q and columns of cluster j is dense.
bool Planner::leaf_is_dense(int32_t q, int32_t j) const {
    const Block *B = root;
    while (B->kind == B_PART) {
        const int32_t r0 = cl[B->t].son0, c0 = cl[B->s].son0;
        const int i = cl[q].begin < cl[r0].begin + cl[r0].size ? 0 : 1;
        const int k = cl[j].begin < cl[c0].begin + cl[c0].size ? 0 : 1;
        B = B->son[i][k];
    }
    return B->kind == B_DENSE;
}

// The largest clusters of order <= bound under t (in a batch, clusters of one problem only: a block
// over several problems would couple their solves through its zero blocks).
void Planner::choose_inverses(int32_t t, int32_t bound) {
    const bool one_problem = inst.empty() || inst[t] >= 0;
    if ((cl[t].size <= bound && one_problem) || cl[t].son0 < 0) {
        inv_index[t] = int32_t(inv_cl.size());
        inv_cl.push_back(t);
        return;
    }
    choose_inverses(cl[t].son0, bound);
    choose_inverses(cl[t].son1, bound);
}

// Y (rows of F->t) := L^{-1} Y where Y is zero in the rows before s0: parts of the recursion that
// only touch those rows are skipped (their result is zero).
void Planner::inv_solve_lower(Block *F, const View &Y, int32_t s0) {
    if (cl[F->t].begin + cl[F->t].size <= s0) return;
    if (F->kind == B_DENSE) {
        Store &s = st(F);
        View D = viewD(F);
        P->trsm.push_back(TTrsm{s.D_off, s.m, TR_LOWER_UNIT | kTrsmNoFlops, Y.p});
        emit(K_TRSM, {&D}, {&Y});
        return;
    }
    const int32_t t0 = cl[F->t].son0, t1 = cl[F->t].son1;
    inv_solve_lower(F->son[0][0], rows(Y, t0), s0);
    if (cl[t0].begin + cl[t0].size > s0) hmm(rows(Y, t1), -1.0, false, F->son[1][0], false, rows(Y, t0));
    inv_solve_lower(F->son[1][1], rows(Y, t1), s0);
}

// Y := U^{-1} Y where Y is zero in the rows from e0 on.
void Planner::inv_solve_upper(Block *F, const View &Y, int32_t e0) {
    if (cl[F->t].begin >= e0) return;
    if (F->kind == B_DENSE) {
        Store &s = st(F);
        View D = viewD(F);
        P->trsm.push_back(TTrsm{s.D_off, s.m, TR_UPPER | kTrsmNoFlops, Y.p});
        emit(K_TRSM, {&D}, {&Y});
        return;
    }
    const int32_t t0 = cl[F->t].son0, t1 = cl[F->t].son1;
    inv_solve_upper(F->son[1][1], rows(Y, t1), e0);
    if (cl[t1].begin < e0) hmm(rows(Y, t0), -1.0, false, F->son[0][1], false, rows(Y, t1));
    inv_solve_upper(F->son[0][0], rows(Y, t0), e0);
}

// Forms L_cc^{-1} and U_cc^{-1} of every inverse block (factorisation plan, after lu(root)).
void Planner::plan_inverses() {
    no_flops = true;
    inv_L_off.assign(inv_cl.size(), 0);
    inv_U_off.assign(inv_cl.size(), 0);
    inv_objL.assign(inv_cl.size(), -1);
    inv_objU.assign(inv_cl.size(), -1);
    for (size_t i = 0; i < inv_cl.size(); ++i) {
        const int32_t c = inv_cl[i], nc = cl[c].size, b0 = cl[c].begin;
        // the diagonal block (c, c) of the block tree
        Block *F = root;
        while (F->t != c) {
            const int32_t s0 = cl[F->t].son0;
            const int side = cl[c].begin < cl[s0].begin + cl[s0].size ? 0 : 1;
            F = F->son[side][side];
        }
        for (int up = 0; up < 2; ++up) {
            const int64_t off = plan_alloc(int64_t(nc) * nc, -1);
            const int32_t obj = new_obj(c, c);
            (up ? inv_U_off : inv_L_off)[i] = off;
            (up ? inv_objU : inv_objL)[i] = obj;
            for (int32_t k = 0; k < cl[c].lc_count; ++k) {
                const int32_t q = lc_ids[cl[c].lc_first + k], mq = cl[q].size, bq = cl[q].begin;
                View Y;
                Y.p = Panel{off + int64_t(bq - b0) * nc, nc, mq, -1, -1, 1, nc};
                Y.obj = obj;
                Y.r_cl = c;
                Y.c_cl = q;
                Y.trans = false;
                // Y = the columns of the identity for the rows of q: one overwrite per leaf cluster
                // of rows (an ACCUM output has at most a leaf cluster's rows), the identity at q
                for (int32_t kk = 0; kk < cl[c].lc_count; ++kk) {
                    const int32_t r = lc_ids[cl[c].lc_first + kk];
                    View Yr = rows(Y, r);
                    if (r == q) {
                        View I = ident(q);
                        P->terms.push_back(Term{I.p, I.p});
                        P->accum.push_back(TAccum{Yr.p, 1.0, 1, int32_t(P->terms.size() - 1), 1, -1, -1, -1.0f});
                        emit(K_ACCUM, {&I}, {&Yr});
                    } else {
                        P->accum.push_back(TAccum{Yr.p, 1.0, 1, int32_t(P->terms.size()), 0, -1, -1, -1.0f});
                        emit(K_ACCUM, {}, {&Yr});
                    }
                }
                if (up)
                    inv_solve_upper(F, Y, bq + mq);
                else
                    inv_solve_lower(F, Y, bq);
            }
        }
    }
    no_flops = false;
}

// out (rows of c) = L_cc^{-1} in or U_cc^{-1} in: one product per leaf cluster q of c over the
// triangle's columns (those of c up to q's end, or from q's start).  The model flops credited are
// the method's own for that row of the substitution: the triangular solve with q's diagonal leaf
// (m_q^2 per column) and the products with the dense leaves of the row inside the block (the
// low-rank ones, of run-time rank, are not credited).
void Planner::apply_inverse(int32_t idx, bool upper, const View &in, const View &out) {
    const int32_t c = inv_cl[idx], nc = cl[c].size, b0 = cl[c].begin, e0 = b0 + nc;
    const int64_t base = upper ? inv_U_off[idx] : inv_L_off[idx];
    const int32_t obj = upper ? inv_objU[idx] : inv_objL[idx];
    std::vector<View> keep;
    std::vector<const View *> rd;
    for (int32_t k = 0; k < cl[c].lc_count; ++k) {
        const int32_t q = lc_ids[cl[c].lc_first + k], mq = cl[q].size, bq = cl[q].begin;
        const int32_t j0 = upper ? bq : b0, j1 = upper ? e0 : bq + mq;  // columns [j0, j1)
        Panel A{base + int64_t(bq - b0) + int64_t(j0 - b0) * nc, mq, j1 - j0, -1, -1, 1, nc};
        Panel X = in.p;
        X.off += int64_t(j0 - b0) * in.p.rs;
        X.rows = j1 - j0;
        X.rslot = -1;
        keep.clear();
        const int32_t k0 = upper ? k : 0, k1 = upper ? cl[c].lc_count : k + 1;
        keep.reserve(2 * (k1 - k0));
        double credit = double(mq) * mq;
        for (int32_t kk = k0; kk < k1; ++kk) {
            const int32_t j = lc_ids[cl[c].lc_first + kk];
            View Lv;
            Lv.p = A;
            Lv.obj = obj;
            Lv.r_cl = q;
            Lv.c_cl = j;
            Lv.trans = false;
            keep.push_back(Lv);
            keep.push_back(rows(in, j));
            if (j != q && leaf_is_dense(q, j)) credit += 2.0 * mq * cl[j].size;
        }
        rd.clear();
        for (const View &v : keep) rd.push_back(&v);
        View o = rows(out, q);
        P->terms.push_back(Term{A, X});
        P->accum.push_back(TAccum{o.p, 1.0, 1, int32_t(P->terms.size() - 1), 1, -1, -1, float(credit)});
        emit(K_ACCUM, rd, {&o});
    }
}

// x = L^{-1} y from Y into Z (Z's rows of F->t are written, Y's are updated in place above the
// inverse level).
void Planner::solve_lower_pp(Block *F, const View &Y, const View &Z) {
    const int32_t idx = inv_index[F->t];
    if (idx >= 0) {
        apply_inverse(idx, false, Y, Z);
        return;
    }
    const int32_t t0 = cl[F->t].son0, t1 = cl[F->t].son1;
    solve_lower_pp(F->son[0][0], rows(Y, t0), rows(Z, t0));
    hmm(rows(Y, t1), -1.0, false, F->son[1][0], false, rows(Z, t0));
    solve_lower_pp(F->son[1][1], rows(Y, t1), rows(Z, t1));
}

// x = U^{-1} z from Z into Y.
void Planner::solve_upper_pp(Block *F, const View &Z, const View &Y) {
    const int32_t idx = inv_index[F->t];
    if (idx >= 0) {
        apply_inverse(idx, true, Z, Y);
        return;
    }
    const int32_t t0 = cl[F->t].son0, t1 = cl[F->t].son1;
    solve_upper_pp(F->son[1][1], rows(Z, t1), rows(Y, t1));
    hmm(rows(Z, t0), -1.0, false, F->son[0][1], false, rows(Y, t1));
    solve_upper_pp(F->son[0][0], rows(Z, t0), rows(Y, t0));
}

// --------------------------------------------------------- plan bookkeeping
void Planner::begin_plan(Plan &p, bool astore_mode, int64_t *bump) {
    dep.pred_mark.clear();
    P = &p;
    use_astore = astore_mode;
    arena = bump;
    std::fill(dep.cell.begin(), dep.cell.end(), CellState{-1, -1, -1, -1});
    dep.rpool_task.clear();
    dep.rpool_next.clear();
    plan_items.clear();  // every plan (and arena) has its own temporaries
    plan_begin = *bump;
    dep.touch_obj.clear();
    dep.touch_cell.clear();
    dep.touch_task.clear();
    dep.touch_write.clear();
    temp_shape.assign(objs.size(), {-1, -1, -1, -1});
    temp_size.assign(objs.size(), 0);
    dep.temp_first.assign(objs.size(), INT32_MAX);
    dep.temp_last.assign(objs.size(), -1);
}

// Sorts a kind's tasks by wave (stable counting sort: waves are small integers); returns the new
// position of every old index.
template <class T>
static std::vector<int32_t> permute_by_wave(std::vector<T> &v, std::vector<int32_t> &w, int32_t n_waves) {
    std::vector<int32_t> start(size_t(n_waves) + 1, 0), where(v.size());
    for (int32_t x : w) start[x + 1]++;
    for (int32_t k = 0; k < n_waves; ++k) start[k + 1] += start[k];
    for (size_t i = 0; i < v.size(); ++i) where[i] = start[w[i]]++;
    std::vector<T> nv(v.size());
    std::vector<int32_t> nw(w.size());
    for (size_t i = 0; i < v.size(); ++i) {
        nv[where[i]] = v[i];
        nw[where[i]] = w[i];
    }
    v.swap(nv);
    w.swap(nw);
    return where;
}

// Rounded-addition scratch of the wave schedule: the tasks of one wave get disjoint regions of the
// arena, waves reuse them (the regions are assigned in emission order within each wave).  The
// data-flow schedule gives every worker its own scratch instead, so nothing is laid out for it.
void Planner::finalize_alloc(Plan &p, int64_t *bump) const {
    const int64_t base = align8(*bump);
    if (!opt.wave_order) {
        for (TRadd &r : p.radd) r.scratch_off = base;
        p.scratch_base = base;
        p.scratch_elems = 0;
        *bump = base;
        return;
    }
    std::vector<int64_t> woff(size_t(std::max(p.n_waves, 1)), 0);
    int64_t maxw = 0;
    for (size_t i = 0; i < p.radd.size(); ++i) {
        TRadd &r = p.radd[i];
        int64_t &off = woff[p.wave[K_RADD][i]];
        r.scratch_off = base + off;
        const int32_t kc = std::min(r.Kcap, opt.kmax_core);
        off = align8(off + int64_t(r.m + r.n) * std::max(kc, 1));
        maxw = std::max(maxw, off);
    }
    p.scratch_base = base;
    p.scratch_elems = maxw;
    *bump = base + maxw;
}

// Orders the tasks by wave, builds the successor lists and priorities and the wave launches.
void Planner::finalize_graph(Plan &p) const {
    std::vector<int32_t> where[K_NKINDS];
    if (opt.wave_order) {
        where[K_GETRF] = permute_by_wave(p.getrf, p.wave[K_GETRF], p.n_waves);
        where[K_TRSM] = permute_by_wave(p.trsm, p.wave[K_TRSM], p.n_waves);
        where[K_PROJECT] = permute_by_wave(p.project, p.wave[K_PROJECT], p.n_waves);
        where[K_ACCUM] = permute_by_wave(p.accum, p.wave[K_ACCUM], p.n_waves);
        where[K_RADD] = permute_by_wave(p.radd, p.wave[K_RADD], p.n_waves);
        where[K_SPLIT] = permute_by_wave(p.split, p.wave[K_SPLIT], p.n_waves);
        // task codes follow the permutation
        for (int32_t &c : p.task_code) {
            const int32_t k = c >> kCodeShift, i = c & kCodeMask;
            c = (k << kCodeShift) | where[k][i];
        }
    }
    // successors from the predecessor lists
    const int64_t nt = p.n_tasks;
    if (p.pred_ptr.empty()) p.pred_ptr.push_back(0);
    p.indeg.assign(nt, 0);
    p.succ_ptr.assign(nt + 1, 0);
    for (int64_t g = 0; g < nt; ++g) {
        p.indeg[g] = p.pred_ptr[g + 1] - p.pred_ptr[g];
        for (int32_t e = p.pred_ptr[g]; e < p.pred_ptr[g + 1]; ++e) p.succ_ptr[p.pred_idx[e] + 1]++;
    }
    for (int64_t g = 0; g < nt; ++g) p.succ_ptr[g + 1] += p.succ_ptr[g];
    p.succ_idx.assign(p.pred_idx.size(), 0);
    {
        std::vector<int32_t> fill(p.succ_ptr.begin(), p.succ_ptr.end() - 1);
        for (int64_t g = 0; g < nt; ++g)
            for (int32_t e = p.pred_ptr[g]; e < p.pred_ptr[g + 1]; ++e) p.succ_idx[fill[p.pred_idx[e]]++] = int32_t(g);
    }
    p.n_edges = (int64_t)p.pred_idx.size();
    // priorities: bottom level (longest path to the end of the graph) with per-kind task latencies
    // measured on the GPU (microseconds: GETRF 27, TRSM 7, PROJECT 3, ACCUM 7, RADD 95, SPLIT 3).
    // The successor on the longest remaining path goes first in every successor list (the
    // data-flow executor prefers the first ready successor), and the roots are sorted by it.
    {
        static const float kLatency[K_NKINDS] = {27.f, 7.f, 3.f, 7.f, 95.f, 3.f};
        std::vector<float> bl(nt, 0.f);
        for (int64_t g = nt - 1; g >= 0; --g) {
            float m = 0.f;
            int32_t best = -1;
            for (int32_t e = p.succ_ptr[g]; e < p.succ_ptr[g + 1]; ++e)
                if (best < 0 || bl[p.succ_idx[e]] > m) {
                    m = bl[p.succ_idx[e]];
                    best = e;
                }
            if (best > p.succ_ptr[g]) std::swap(p.succ_idx[best], p.succ_idx[p.succ_ptr[g]]);
            bl[g] = m + kLatency[p.task_code[g] >> kCodeShift];
        }
        auto by_priority = [&](int32_t x, int32_t y) { return bl[x] > bl[y] || (bl[x] == bl[y] && x < y); };
        p.roots.clear();
        p.critical_us = 0.0;
        for (int64_t g = 0; g < nt; ++g)
            if (p.indeg[g] == 0) {
                p.roots.push_back(int32_t(g));
                p.critical_us = std::max(p.critical_us, double(bl[g]));
            }
        std::sort(p.roots.begin(), p.roots.end(), by_priority);
        p.root_bl.resize(p.roots.size());
        for (size_t r = 0; r < p.roots.size(); ++r) p.root_bl[r] = bl[p.roots[r]];
    }
    // launches: for each wave, one launch per kind present (wave order only)
    if (!opt.wave_order) return;
    size_t pos[K_NKINDS] = {0, 0, 0, 0, 0, 0};
    for (int32_t w = 0; w < p.n_waves; ++w) {
        for (int k = 0; k < K_NKINDS; ++k) {
            std::vector<int32_t> &wv = p.wave[k];
            size_t s = pos[k];
            while (pos[k] < wv.size() && wv[pos[k]] == w) ++pos[k];
            if (pos[k] > s) p.launches.push_back(Launch{w, k, int32_t(s), int32_t(pos[k] - s)});
        }
    }
}

// ------------------------------------------------------------- validation
int Planner::build_tree() {
    std::map<std::pair<int32_t, int32_t>, int64_t> idx;
    for (int64_t l = 0; l < n_leaves; ++l) {
        auto key = std::make_pair(leaf_row[l], leaf_col[l]);
        if (idx.count(key)) {
            error = "duplicate leaf block";
            return HLU_EINVAL;
        }
        idx[key] = l;
    }
    int64_t used = 0;
    std::vector<std::pair<Block **, std::pair<int32_t, int32_t>>> stack;
    stack.push_back({&root, {0, 0}});
    while (!stack.empty()) {
        auto it = stack.back();
        stack.pop_back();
        int32_t t = it.second.first, s = it.second.second;
        Block *b = new Block{t, s, B_PART, -1, {{nullptr, nullptr}, {nullptr, nullptr}}};
        blocks_owned.push_back(b);
        *it.first = b;
        auto f = idx.find({t, s});
        if (f != idx.end()) {
            int64_t l = f->second;
            b->kind = leaf_kind[l] == 0 ? B_DENSE : B_LOWRANK;
            b->id = int32_t(l);
            if (t == s && b->kind == B_LOWRANK) {
                error = "low-rank diagonal block";
                return HLU_EINVAL;
            }
            if (b->kind == B_DENSE && cl[t].son0 >= 0 && cl[s].son0 >= 0) {
                // Algorithm 2 partitions a non-admissible block whose clusters both have sons
                error = "dense leaf between two clusters that both have sons";
                return HLU_EINVAL;
            }
            used++;
            continue;
        }
        if (!inst.empty() && (inst[t] != inst[s] || (t != s && inst[t] < 0))) {
            b->kind = B_ZERO;  // between two instances of a batch
            continue;
        }
        if (cl[t].son0 < 0 || cl[s].son0 < 0) {
            error = "leaves do not tile the matrix (missing block)";
            return HLU_EINVAL;
        }
        int32_t ts[2] = {cl[t].son0, cl[t].son1}, ss[2] = {cl[s].son0, cl[s].son1};
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) stack.push_back({&b->son[i][j], {ts[i], ss[j]}});
    }
    if (used != n_leaves) {
        error = "leaves do not tile the matrix (overlapping or unreachable leaf)";
        return HLU_EINVAL;
    }
    return HLU_OK;
}

void Planner::layout_factor_arena() {
    f_elems = 0;
    fstore.assign(n_leaves, Store{});
    for (int64_t l = 0; l < n_leaves; ++l) {
        Store &s = fstore[l];
        s.t = leaf_row[l];
        s.s = leaf_col[l];
        s.m = cl[s.t].size;
        s.n = cl[s.s].size;
        s.krank = leaf_rank[l];
        s.objD = s.objU = s.objV = -1;
        if (leaf_kind[l] == 0) {
            s.kind = B_DENSE;
            s.D_off = f_elems;
            f_elems = align8(f_elems + int64_t(s.m) * s.n);
            s.objD = new_obj(s.t, s.s);
            s.kslot = -1;
            s.cap = 0;
        } else {
            s.kind = B_LOWRANK;
            s.cap = std::min(std::min(s.m, s.n), std::max(opt.rank_cap, s.krank));
            s.U_off = f_elems;
            f_elems = align8(f_elems + int64_t(s.m) * s.cap);
            s.V_off = f_elems;
            f_elems = align8(f_elems + int64_t(s.n) * s.cap);
            s.kslot = new_slot(s.krank);
            s.objU = new_obj(s.t, -1);
            s.objV = new_obj(s.s, -1);
        }
    }
    f_ident_off = f_elems;
    f_elems = align8(f_elems + int64_t(max_leaf) * max_leaf);
    ident_obj = new_obj(-1, -1);
}

void Planner::layout_a_arena() {
    a_elems = 0;
    astore.assign(n_leaves, Store{});
    for (int64_t l = 0; l < n_leaves; ++l) {
        Store &s = astore[l];
        s = fstore[l];
        s.kslot = -1;
        s.cap = s.krank;
        if (s.kind == B_DENSE) {
            s.D_off = a_elems;
            a_elems = align8(a_elems + int64_t(s.m) * s.n);
            s.objD = new_obj(s.t, s.s);
        } else {
            s.U_off = a_elems;
            a_elems = align8(a_elems + int64_t(s.m) * s.krank);
            s.V_off = a_elems;
            a_elems = align8(a_elems + int64_t(s.n) * s.krank);
            s.objU = new_obj(s.t, -1);
            s.objV = new_obj(s.s, -1);
        }
    }
}

int Planner::build(int32_t n_, int32_t n_clusters, const int32_t *perm_, const int32_t *begin,
                   const int32_t *size, const int32_t *son0, const int32_t *son1, int64_t n_leaves_,
                   const int32_t *row_cl, const int32_t *col_cl, const int8_t *kind,
                   const int32_t *rank, const int64_t *offset, const double *data,
                   int64_t data_len, const PlanOptions &o, const int32_t *inst_, int32_t n_inst_) {
    opt = o;
    n = n_;
    inst.clear();
    n_inst = 1;
    if (inst_) {
        if (n_inst_ < 1) {
            error = "bad instance count";
            return HLU_EINVAL;
        }
        inst.assign(inst_, inst_ + n_clusters);
        for (int32_t v : inst)
            if (v < -1 || v >= n_inst_) {
                error = "bad instance index";
                return HLU_EINVAL;
            }
        n_inst = n_inst_;
    }
    if (n < 1 || n_clusters < 1 || !perm_ || !begin || !size || !son0 || !son1) {
        error = "bad tree arguments";
        return HLU_EINVAL;
    }
    cl.resize(n_clusters);
    for (int32_t c = 0; c < n_clusters; ++c) {
        cl[c].begin = begin[c];
        cl[c].size = size[c];
        cl[c].son0 = son0[c];
        cl[c].son1 = son1[c];
        cl[c].lc_first = cl[c].lc_count = 0;
        if (size[c] < 1 || begin[c] < 0 || int64_t(begin[c]) + size[c] > n) {
            error = "cluster range outside [0, n)";
            return HLU_EINVAL;
        }
        bool l0 = son0[c] < 0, l1 = son1[c] < 0;
        if (l0 != l1) {
            error = "cluster with exactly one son";
            return HLU_EINVAL;
        }
        if (!l0) {
            if (son0[c] >= n_clusters || son1[c] >= n_clusters || son0[c] == 0 || son1[c] == 0 ||
                son0[c] == son1[c]) {
                error = "bad son index";
                return HLU_EINVAL;
            }
        }
    }
    if (cl[0].begin != 0 || cl[0].size != n) {
        error = "root cluster must cover [0, n)";
        return HLU_EINVAL;
    }
    // walk the tree: check son ranges, count visits, number leaf clusters in DoF order
    std::vector<int32_t> visits(n_clusters, 0);
    std::vector<int32_t> stack{0};
    std::vector<int32_t> order;
    while (!stack.empty()) {
        int32_t c = stack.back();
        stack.pop_back();
        if (visits[c]++) {
            error = "cluster reached twice (not a tree)";
            return HLU_EINVAL;
        }
        order.push_back(c);
        if (cl[c].son0 >= 0) {
            const ClusterInfo &a = cl[cl[c].son0], &b = cl[cl[c].son1];
            if (a.begin != cl[c].begin || b.begin != cl[c].begin + a.size || a.size + b.size != cl[c].size) {
                error = "son ranges do not split the parent";
                return HLU_EINVAL;
            }
            stack.push_back(cl[c].son1);
            stack.push_back(cl[c].son0);
        }
    }
    if ((int32_t)order.size() != n_clusters) {
        error = "unreachable cluster";
        return HLU_EINVAL;
    }
    // leaf clusters in DoF order (pre-order with son0 first is DoF order)
    lc_ids.clear();
    max_leaf = 0;
    for (int32_t c : order)
        if (cl[c].son0 < 0) {
            cl[c].lc_first = int32_t(lc_ids.size());
            cl[c].lc_count = 1;
            lc_ids.push_back(c);
            max_leaf = std::max(max_leaf, cl[c].size);
        }
    if (max_leaf > kMaxLeafRows) {
        error = "leaf cluster larger than 128 indices";
        return HLU_EINVAL;
    }
    for (auto it = order.rbegin(); it != order.rend(); ++it) {
        int32_t c = *it;
        if (cl[c].son0 >= 0) {
            cl[c].lc_first = cl[cl[c].son0].lc_first;
            cl[c].lc_count = cl[cl[c].son0].lc_count + cl[cl[c].son1].lc_count;
        }
    }
    perm.assign(perm_, perm_ + n);
    {
        std::vector<char> seen(n, 0);
        for (int32_t p : perm) {
            if (p < 0 || p >= n || seen[p]) {
                error = "perm is not a permutation";
                return HLU_EINVAL;
            }
            seen[p] = 1;
        }
    }
    n_leaves = n_leaves_;
    if (n_leaves < 1 || !row_cl || !col_cl || !kind || !rank || !offset || !data) {
        error = "bad block arguments";
        return HLU_EINVAL;
    }
    leaf_row.assign(row_cl, row_cl + n_leaves);
    leaf_col.assign(col_cl, col_cl + n_leaves);
    leaf_kind.assign(kind, kind + n_leaves);
    leaf_rank.assign(rank, rank + n_leaves);
    leaf_offset.assign(offset, offset + n_leaves);
    for (int64_t l = 0; l < n_leaves; ++l) {
        if (leaf_row[l] < 0 || leaf_row[l] >= n_clusters || leaf_col[l] < 0 || leaf_col[l] >= n_clusters) {
            error = "leaf cluster index out of range";
            return HLU_EINVAL;
        }
        if (leaf_kind[l] != 0 && leaf_kind[l] != 1) {
            error = "leaf kind must be 0 or 1";
            return HLU_EINVAL;
        }
        int32_t m = cl[leaf_row[l]].size, nn = cl[leaf_col[l]].size;
        if (leaf_kind[l] == 1 && (leaf_rank[l] < 0 || leaf_rank[l] > std::min(m, nn))) {
            error = "rank outside [0, min(m, n)]";
            return HLU_EINVAL;
        }
        int64_t len = leaf_kind[l] == 0 ? int64_t(m) * nn : int64_t(m + nn) * leaf_rank[l];
        if (leaf_offset[l] < 0 || leaf_offset[l] + len > data_len) {
            error = "leaf data outside the data array";
            return HLU_EINVAL;
        }
    }
    // every value a leaf covers must be finite: an exponent field of all ones is an infinity or a
    // NaN.  A vectorisable scan, split over host threads by leaves (the data can be GBs).
    auto scan = [&](int64_t l0, int64_t l1) {
        uint64_t bad = 0;
        for (int64_t l = l0; l < l1; ++l) {
            const int32_t m = cl[leaf_row[l]].size, nn = cl[leaf_col[l]].size;
            const int64_t len = leaf_kind[l] == 0 ? int64_t(m) * nn : int64_t(m + nn) * leaf_rank[l];
            const double *dl = data + leaf_offset[l];
            for (int64_t i = 0; i < len; ++i) {
                uint64_t bits;
                std::memcpy(&bits, dl + i, sizeof(bits));
                bad |= uint64_t((bits & 0x7ff0000000000000ull) == 0x7ff0000000000000ull);
            }
        }
        return bad != 0;
    };
    const int nthreads = int(std::min<int64_t>(std::max(1u, std::min(8u, std::thread::hardware_concurrency())),
                                                std::max<int64_t>(1, n_leaves / 256)));
    bool bad = false;
    if (nthreads <= 1) {
        bad = scan(0, n_leaves);
    } else {
        std::vector<char> flag(nthreads, 0);
        run_parts(nthreads, [&](int q) { flag[q] = scan(n_leaves * q / nthreads, n_leaves * (q + 1) / nthreads); });
        for (char f : flag) bad = bad || f;
    }
    if (bad) {
        error = "non-finite input value";
        return HLU_EINVAL;
    }
    if (n_inst > 1 && !opt.wave_order && opt.batch_threads >= 0) {
        batch_deferred = true;  // every problem gets its own block tree in plan_batch
        return HLU_OK;
    }
    return build_tree();
}

// Capacity for the factorisation plan's lists from an estimate of its task count (about 7 to 10
// tasks per leaf per level of the cluster tree on surface meshes), so that they are not copied as
// they grow; capacity that is not used is never touched.
void Planner::reserve_factorisation() {
    int32_t depth = 1;
    for (int64_t c = cl[0].lc_count; c > 1; c = (c + 1) / 2) ++depth;
    const int64_t t = std::min<int64_t>(int64_t(n_leaves) * 10 * depth, int64_t(1) << 25);  // larger plans grow past it
    Plan &p = fplan;
    p.task_code.reserve(size_t(t));
    p.getrf.reserve(size_t(cl[0].lc_count));
    p.wave[K_GETRF].reserve(size_t(cl[0].lc_count));
    const double share[K_NKINDS] = {0.0, 0.1, 0.3, 0.6, 0.25, 0.05};
    for (int k = K_TRSM; k < K_NKINDS; ++k) p.wave[k].reserve(size_t(share[k] * double(t)));
    p.trsm.reserve(size_t(share[K_TRSM] * double(t)));
    p.project.reserve(size_t(share[K_PROJECT] * double(t)));
    p.accum.reserve(size_t(share[K_ACCUM] * double(t)));
    p.radd.reserve(size_t(share[K_RADD] * double(t)));
    p.split.reserve(size_t(share[K_SPLIT] * double(t)));
    p.terms.reserve(size_t(t));
    p.pieces.reserve(size_t(0.25 * double(t)));
    p.pred_ptr.reserve(size_t(t) + 1);
    p.pred_idx.reserve(size_t(5 * t));
    const size_t nobj = objs.size() + size_t(0.4 * double(t));
    objs.reserve(nobj);
    plan_items.reserve(size_t(0.4 * double(t)));
    temp_size.reserve(nobj);
    temp_shape.reserve(nobj);
    dep.temp_first.reserve(nobj);
    dep.temp_last.reserve(nobj);
    dep.cell.reserve(2 * nobj);
    dep.pred_mark.reserve(size_t(2 * t));
    dep.rpool_task.reserve(size_t(6 * t));
    dep.rpool_next.reserve(size_t(6 * t));
}

int Planner::plan_all() {
    if (batch_deferred) return plan_batch();
    layout_factor_arena();
    nrhs_slot = new_slot(0);
    begin_plan(fplan, false, &f_elems);
    auto emit_factorisation = [&] {
        lu(root);
        inv_cl.clear();
        inv_index.assign(cl.size(), -1);
        if (opt.inv_block > 0) {
            choose_inverses(0, std::max(opt.inv_block, max_leaf));
            plan_inverses();
        }
    };
    reserve_factorisation();
    // one plan of one piece: the dependency analysis of the factorisation on a second thread, and its
    // graph finished (successors, priorities) while the solve and the matvec are emitted
    const bool piped = opt.batch_threads >= 0 && std::thread::hardware_concurrency() > 1 && pipe_begin();
    if (piped) {
        bool oom = false;
        try {
            emit_factorisation();
        } catch (const std::bad_alloc &) {
            oom = true;
        }
        const int st = pipe_end();
        if (oom) {
            error = "out of host memory while emitting the factorisation";
            return HLU_ENOMEM;
        }
        if (st != HLU_OK) return st;
    } else {
        emit_factorisation();
    }
    dep.temp_first.resize(temp_size.size(), INT32_MAX);
    dep.temp_last.resize(temp_size.size(), -1);
    temp_levels(fplan);
    if (opt.temp_reuse) relocate_temps(fplan);
    finalize_alloc(fplan, &f_elems);
    struct Joiner {
        std::thread th;
        ~Joiner() {
            if (th.joinable()) th.join();
        }
    } fgraph;
    if (piped) {
        try {
            fgraph.th = std::thread([this] { finalize_graph(fplan); });
        } catch (const std::system_error &) {
            finalize_graph(fplan);
        }
    } else {
        finalize_graph(fplan);
    }
    f_solve_off = f_elems;
    f_elems = align8(f_elems + int64_t(n) * opt.nrhs_max);
    View Y;
    Y.p = Panel{f_solve_off, n, opt.nrhs_max, -1, nrhs_slot, 1, n};
    Y.obj = new_obj(0, -1);
    Y.r_cl = 0;
    Y.c_cl = -1;
    Y.trans = false;
    begin_plan(splan, false, &f_elems);
    split_accum = true;
    if (!inv_cl.empty()) {
        f_z_off = f_elems;
        f_elems = align8(f_elems + int64_t(n) * opt.nrhs_max);
        View Z = Y;
        Z.p.off = f_z_off;
        Z.obj = new_obj(0, -1);
        solve_lower_pp(root, Y, Z);
        solve_upper_pp(root, Z, Y);
    } else {
        solve_lower(root, Y);
        solve_upper(root, Y);
    }
    split_accum = false;
    finalize_alloc(splan, &f_elems);
    finalize_graph(splan);
    layout_a_arena();
    a_x_off = a_elems;
    a_elems = align8(a_elems + int64_t(n) * opt.nrhs_max);
    a_y_off = a_elems;
    a_elems = align8(a_elems + int64_t(n) * opt.nrhs_max);
    View X = Y, Yo = Y;
    X.p.off = a_x_off;
    X.obj = new_obj(0, -1);
    Yo.p.off = a_y_off;
    Yo.obj = new_obj(0, -1);
    begin_plan(mplan, true, &a_elems);
    hmm(Yo, 1.0, true, root, false, X);
    finalize_alloc(mplan, &a_elems);
    finalize_graph(mplan);
    if (fgraph.th.joinable()) fgraph.th.join();
    P = nullptr;
    // the ACCUM kernel keeps one output row per thread slot (at most 1024 rows)
    for (const Plan *pp : {&fplan, &splan, &mplan})
        for (const TAccum &t : pp->accum)
            if (t.out.rows > 1024) {
                error = "internal: product output with more than 1024 rows";
                return HLU_EINVAL;
            }
    return HLU_OK;
}

}  // namespace hlu
