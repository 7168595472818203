// Planning of a batch of independent H-matrices on several host threads.
//
// The problems of a batch share no block, no task and no dependency: the LU recursion of Sec. 3.1
// on the block-diagonal forest only ever descends into the diagonal blocks of single problems (the
// blocks between two problems are structurally zero).  So every problem is planned on its own, by
// its own Planner on a thread of a pool, and the per-problem task graphs are joined afterwards:
// each problem's arena region, dynamic-dimension slots, block ids, cluster ids, task indices and
// dependency edges are shifted by the sums over the problems before it.  Three regions are shared
// by the whole batch instead of being per problem: the n x nrhs_max work panels of the solve (and
// of the inverse-block solve) and of the matrix-vector product, which the caller fills and reads
// as one stacked system (a problem's rows at its offset, leading dimension n), and the identity
// block of the largest leaf.  Views into a problem's own copy of those regions move to the shared
// one with the leading dimension changed; the per-problem copies stay unused in the arena.
//
// The joined graph has the tasks and edges the single plan of the whole forest has (the same
// recursion per problem, and no cell is written by two problems).
#include <algorithm>
#include <atomic>
#include <memory>
#include <new>
#include <thread>

#include "../../include/hlu.h"
#include "plan.h"

namespace hlu {

namespace {

inline int64_t align8(int64_t x) { return (x + 7) & ~int64_t(7); }

// A column-major region of one problem's arena that moves to a shared region of the batch:
// element (r, c) at base + r + c * ld goes to nbase + r + c * nld.
struct Moved {
    int64_t base, len;
    int32_t ld;
    int64_t nbase;
    int32_t nld;
};

// Where one problem's plan goes in the joined plan.
struct Shift {
    int64_t arena = 0;               // offset of the problem's arena region
    std::vector<Moved> moved;        // regions that move to the shared panels instead
    int32_t slot = 0;                // first dynamic-dimension slot
    int32_t own_nrhs = -1, nrhs = -1;  // the problem's panel-width slot and the batch's
    int32_t cluster = 0;             // first cluster in the forest numbering
    int32_t leaf = 0, n_leaves = 0;  // first input leaf, the problem's input leaves
    int32_t split = 0;               // first temporary split block (store id)
    int32_t inst = 0;

    int64_t off(int64_t o) const {
        for (const Moved &m : moved)
            if (o >= m.base && o < m.base + m.len) {
                const int64_t loc = o - m.base;
                return m.nbase + loc % m.ld + (loc / m.ld) * m.nld;
            }
        return o + arena;
    }
    void panel(Panel &p) const {
        for (const Moved &m : moved)
            if (p.off >= m.base && p.off < m.base + m.len) {
                const int64_t loc = p.off - m.base;
                p.off = m.nbase + loc % m.ld + (loc / m.ld) * m.nld;
                if (p.rs == m.ld) p.rs = m.nld;
                if (p.cs == m.ld) p.cs = m.nld;
                p.rslot = slot_of(p.rslot);
                p.cslot = slot_of(p.cslot);
                return;
            }
        p.off += arena;
        p.rslot = slot_of(p.rslot);
        p.cslot = slot_of(p.cslot);
    }
    int32_t slot_of(int32_t s) const { return s < 0 ? s : s == own_nrhs ? nrhs : s + slot; }
    int32_t store(int32_t id) const { return id < n_leaves ? id + leaf : id - n_leaves + split; }
};

// Bases of one plan of one problem in the joined plan.
struct PlanBase {
    int64_t kind[K_NKINDS] = {0, 0, 0, 0, 0, 0};
    int64_t terms = 0, pieces = 0, tasks = 0, edges = 0, roots = 0;
};

void add_sizes(const Plan &p, PlanBase &b) {
    b.kind[K_GETRF] += (int64_t)p.getrf.size();
    b.kind[K_TRSM] += (int64_t)p.trsm.size();
    b.kind[K_PROJECT] += (int64_t)p.project.size();
    b.kind[K_ACCUM] += (int64_t)p.accum.size();
    b.kind[K_RADD] += (int64_t)p.radd.size();
    b.kind[K_SPLIT] += (int64_t)p.split.size();
    b.terms += (int64_t)p.terms.size();
    b.pieces += (int64_t)p.pieces.size();
    b.tasks += p.n_tasks;
    b.edges += (int64_t)p.succ_idx.size();
    b.roots += (int64_t)p.roots.size();
}

// Figures of the joined graph: the problems' graphs side by side.
struct Joined {
    int32_t n_waves = 0, max_kcap = 0;
    double critical_us = 0.0;
    int64_t temp_elems = 0, temp_peak_elems = 0;
    void add(const Plan &p) {
        n_waves = std::max(n_waves, p.n_waves);
        max_kcap = std::max(max_kcap, p.max_kcap);
        critical_us = std::max(critical_us, p.critical_us);
        temp_elems += p.temp_elems;
        temp_peak_elems += p.temp_peak_elems;  // an upper bound: the levels of two problems need not meet
    }
};

// Capacity for the joined plan; the problems' plans are appended in problem order (pages are
// touched only as they are filled, while every problem's own plan is freed after its append, so
// the host holds about one copy of the plans at any time).
void reserve_joined(Plan &q, const PlanBase &tot) {
    q.getrf.reserve(tot.kind[K_GETRF]);
    q.trsm.reserve(tot.kind[K_TRSM]);
    q.project.reserve(tot.kind[K_PROJECT]);
    q.accum.reserve(tot.kind[K_ACCUM]);
    q.radd.reserve(tot.kind[K_RADD]);
    q.split.reserve(tot.kind[K_SPLIT]);
    for (int k = 0; k < K_NKINDS; ++k) q.wave[k].reserve(tot.kind[k]);
    q.terms.reserve(tot.terms);
    q.pieces.reserve(tot.pieces);
    q.task_code.reserve(tot.tasks);
    q.indeg.reserve(tot.tasks);
    q.succ_ptr.reserve(tot.tasks + 1);  // (the predecessor lists, used only while planning, are not kept)
    q.succ_ptr.push_back(0);
    q.succ_idx.reserve(tot.edges);
    q.roots.reserve(tot.roots);
    q.root_bl.reserve(tot.roots);
    q.n_tasks = tot.tasks;
    q.n_edges = tot.edges;
}

// Appends one group of the arrays of problem plan p (bases b: the sizes of the joined arrays so far)
// to the joined plan q, shifting everything by s, and frees them in p.  The groups touch disjoint
// arrays, so they are joined on kJoinGroups threads at once: 0: GETRF, TRSM, PROJECT and SPLIT
// tasks; 1: ACCUM tasks; 2: their terms; 3: RADD tasks and their pieces; 4: the graph (task codes,
// in-degrees, successors, roots).
constexpr int kJoinGroups = 5;

template <class V>
void release(V &v) {
    V().swap(v);
}

void join_group(int group, Plan &p, const PlanBase &b, const Shift &s, Plan &q) {
    auto waves = [&](int k) {
        q.wave[k].insert(q.wave[k].end(), p.wave[k].begin(), p.wave[k].end());
        release(p.wave[k]);
    };
    if (group == 0) {
        for (TGetrf t : p.getrf) {
            t.off = s.off(t.off);
            t.leaf = s.store(t.leaf);
            q.getrf.push_back(t);
        }
        for (TTrsm t : p.trsm) {
            t.L_off = s.off(t.L_off);
            s.panel(t.P);
            q.trsm.push_back(t);
        }
        for (TProject t : p.project) {
            s.panel(t.F);
            s.panel(t.X);
            s.panel(t.T);
            t.dst0 = s.slot_of(t.dst0);
            t.src0 = s.slot_of(t.src0);
            t.dst1 = s.slot_of(t.dst1);
            t.src1 = s.slot_of(t.src1);
            q.project.push_back(t);
        }
        for (TSplit t : p.split) {
            s.panel(t.srcU);
            s.panel(t.srcV);
            t.dstU = s.off(t.dstU);
            t.dstV = s.off(t.dstV);
            t.src_kslot = s.slot_of(t.src_kslot);
            t.dst_kslot = s.slot_of(t.dst_kslot);
            q.split.push_back(t);
        }
        release(p.getrf);
        release(p.trsm);
        release(p.project);
        release(p.split);
        for (int k : {K_GETRF, K_TRSM, K_PROJECT, K_SPLIT}) waves(k);
    } else if (group == 1) {
        for (TAccum t : p.accum) {
            s.panel(t.out);
            t.term0 += int32_t(b.terms);
            t.dst = s.slot_of(t.dst);
            t.src = s.slot_of(t.src);
            q.accum.push_back(t);
        }
        release(p.accum);
        waves(K_ACCUM);
    } else if (group == 2) {
        for (Term t : p.terms) {
            s.panel(t.A);
            s.panel(t.X);
            q.terms.push_back(t);
        }
        release(p.terms);
    } else if (group == 3) {
        for (TRadd t : p.radd) {
            t.U_off = s.off(t.U_off);
            t.V_off = s.off(t.V_off);
            t.scratch_off = s.off(t.scratch_off);
            t.kslot = s.slot_of(t.kslot);
            t.piece0 += int32_t(b.pieces);
            t.target = s.store(t.target);
            t.inst = s.inst;
            q.radd.push_back(t);
        }
        for (Piece t : p.pieces) {
            s.panel(t.U);
            s.panel(t.V);
            q.pieces.push_back(t);
        }
        release(p.radd);
        release(p.pieces);
        waves(K_RADD);
    } else {
        for (int64_t g = 0; g < p.n_tasks; ++g) {
            const int32_t c = p.task_code[g], k = c >> kCodeShift;
            q.task_code.push_back((k << kCodeShift) | int32_t((c & kCodeMask) + b.kind[k]));
            q.indeg.push_back(p.indeg[g]);
            q.succ_ptr.push_back(int32_t(p.succ_ptr[g + 1] + b.edges));
        }
        for (int32_t t : p.succ_idx) q.succ_idx.push_back(int32_t(t + b.tasks));
        for (size_t r = 0; r < p.roots.size(); ++r) {
            q.roots.push_back(int32_t(p.roots[r] + b.tasks));
            q.root_bl.push_back(p.root_bl[r]);
        }
        release(p.task_code);
        release(p.indeg);
        release(p.succ_ptr);
        release(p.succ_idx);
    }
}

}  // namespace

// Instance layout of the forest (as hlu_create_batch builds it): the clusters of every problem
// contiguous and in problem order after the clusters above the problems, each problem's root
// first and covering its rows, rows and leaves contiguous in problem order, every leaf inside one
// problem.  Returns false when the forest is not of that form (it is then planned as one).
bool Planner::batch_layout(std::vector<int32_t> &cb, std::vector<int32_t> &ce, std::vector<int64_t> &lb,
                           std::vector<int32_t> &rb) const {
    const int32_t ncl = (int32_t)cl.size();
    cb.assign(n_inst, -1);
    ce.assign(n_inst, -1);
    int32_t cur = -1;
    for (int32_t c = 0; c < ncl; ++c) {
        const int32_t i = inst[c];
        if (i < 0) {
            if (cur >= 0) return false;  // a cluster above the problems after a problem's clusters
            continue;
        }
        if (i != cur) {
            if (i != cur + 1) return false;
            cb[i] = c;
            cur = i;
        }
        ce[i] = c + 1;
    }
    if (cur != n_inst - 1) return false;
    rb.assign(n_inst + 1, 0);
    for (int32_t i = 0; i < n_inst; ++i) {
        const ClusterInfo &r = cl[cb[i]];
        if (r.begin != rb[i]) return false;
        rb[i + 1] = r.begin + r.size;
        // the problem's clusters are exactly the subtree of its root
        int32_t seen = 0;
        std::vector<int32_t> stack{cb[i]};
        while (!stack.empty()) {
            const int32_t c = stack.back();
            stack.pop_back();
            if (c < cb[i] || c >= ce[i] || ++seen > ce[i] - cb[i]) return false;
            if (cl[c].son0 >= 0) {
                stack.push_back(cl[c].son0);
                stack.push_back(cl[c].son1);
            }
        }
        if (seen != ce[i] - cb[i]) return false;
        for (int32_t k = rb[i]; k < rb[i + 1]; ++k)
            if (perm[k] < rb[i] || perm[k] >= rb[i + 1]) return false;
    }
    if (rb[n_inst] != n) return false;
    lb.assign(n_inst + 1, 0);
    int32_t li = 0;
    for (int64_t l = 0; l < n_leaves; ++l) {
        const int32_t i = inst[leaf_row[l]];
        if (i < 0 || inst[leaf_col[l]] != i || i < li) return false;
        while (li < i) lb[++li] = l;
    }
    while (li < n_inst) lb[++li] = n_leaves;
    return true;
}

int Planner::plan_batch() {
    batch_deferred = false;
    std::vector<int32_t> cb, ce, rb;
    std::vector<int64_t> lb;
    if (!batch_layout(cb, ce, lb, rb)) {  // not the layout of hlu_create_batch: one plan of the forest
        const int st = build_tree();
        return st ? st : plan_all();
    }
    const int32_t count = n_inst;
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const int32_t nthreads = std::max(1, std::min<int32_t>(count, opt.batch_threads > 0 ? opt.batch_threads
                                                                                         : int32_t(hw)));
    // a problem's own dependency analysis gets a second thread when the pool leaves one per problem
    const int32_t part_threads = 2 * nthreads <= int32_t(hw) ? 0 : -1;
    std::vector<std::unique_ptr<Planner>> parts(count);
    for (int32_t i = 0; i < count; ++i) {
        parts[i].reset(new (std::nothrow) Planner());
        if (!parts[i]) return HLU_ENOMEM;
        Planner &q = *parts[i];
        q.opt = opt;
        q.opt.batch_threads = part_threads;
        q.n = rb[i + 1] - rb[i];
        q.n_inst = 1;
        const int32_t c0 = cb[i], lc0 = cl[c0].lc_first;
        q.cl.assign(cl.begin() + c0, cl.begin() + ce[i]);
        for (ClusterInfo &c : q.cl) {
            c.begin -= rb[i];
            if (c.son0 >= 0) {
                c.son0 -= c0;
                c.son1 -= c0;
            }
            c.lc_first -= lc0;
        }
        q.lc_ids.assign(lc_ids.begin() + lc0, lc_ids.begin() + lc0 + cl[c0].lc_count);
        q.max_leaf = 0;
        for (int32_t &c : q.lc_ids) {
            c -= c0;
            q.max_leaf = std::max(q.max_leaf, q.cl[c].size);
        }
        q.perm.assign(perm.begin() + rb[i], perm.begin() + rb[i + 1]);
        for (int32_t &v : q.perm) v -= rb[i];
        q.n_leaves = lb[i + 1] - lb[i];
        q.leaf_row.assign(leaf_row.begin() + lb[i], leaf_row.begin() + lb[i + 1]);
        q.leaf_col.assign(leaf_col.begin() + lb[i], leaf_col.begin() + lb[i + 1]);
        for (int32_t &c : q.leaf_row) c -= c0;
        for (int32_t &c : q.leaf_col) c -= c0;
        q.leaf_kind.assign(leaf_kind.begin() + lb[i], leaf_kind.begin() + lb[i + 1]);
        q.leaf_rank.assign(leaf_rank.begin() + lb[i], leaf_rank.begin() + lb[i + 1]);
        q.leaf_offset.assign(leaf_offset.begin() + lb[i], leaf_offset.begin() + lb[i + 1]);
    }
    // plan the problems on a pool of threads, the largest first
    std::vector<int32_t> order(count);
    for (int32_t i = 0; i < count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t a, int32_t b) { return parts[a]->n_leaves > parts[b]->n_leaves; });
    std::vector<int> status(count, HLU_OK);
    std::atomic<int32_t> next{0};
    auto worker = [&] {
        for (;;) {
            const int32_t j = next.fetch_add(1);
            if (j >= count) return;
            Planner &q = *parts[order[j]];
            int st;
            try {
                st = q.build_tree();
                if (st == HLU_OK) st = q.plan_all();
            } catch (const std::bad_alloc &) {
                st = HLU_ENOMEM;
                q.error = "host memory exhausted while planning";
            }
            q.release_work();
            status[order[j]] = st;
        }
    };
    run_parts(nthreads, [&](int) { worker(); });
    for (int32_t i = 0; i < count; ++i)
        if (status[i] != HLU_OK) {
            error = "problem " + std::to_string(i) + ": " + parts[i]->error;
            return status[i];
        }
    // bases: arena regions, slots, store ids, inverse blocks, and per plan the task arrays
    const int64_t W = opt.nrhs_max;
    std::vector<Shift> fs(count), as(count);
    std::vector<PlanBase> fb(count), sb(count), mb(count);
    PlanBase ft, st_, mt;
    int64_t fpos = 0, apos = 0, nsplit = 0, ninv = 0;
    int32_t nslot = 0;
    bool any_z = false;
    std::vector<int64_t> inv_base(count);
    Joined joined[3];
    for (int32_t i = 0; i < count; ++i) {
        const Planner &q = *parts[i];
        fs[i].arena = fpos;
        as[i].arena = apos;
        fpos = align8(fpos + q.f_elems);
        apos = align8(apos + q.a_elems);
        for (Shift *s : {&fs[i], &as[i]}) {
            s->slot = nslot;
            s->own_nrhs = q.nrhs_slot;
            s->cluster = cb[i];
            s->leaf = int32_t(lb[i]);
            s->n_leaves = int32_t(q.n_leaves);
            s->split = int32_t(n_leaves + nsplit);
            s->inst = i;
        }
        nslot += q.n_slots;
        nsplit += (int64_t)q.fstore.size() - q.n_leaves;
        inv_base[i] = ninv;
        ninv += (int64_t)q.inv_cl.size();
        any_z = any_z || q.f_z_off >= 0;
        fb[i] = ft;
        sb[i] = st_;
        mb[i] = mt;
        add_sizes(q.fplan, ft);
        add_sizes(q.splan, st_);
        add_sizes(q.mplan, mt);
        joined[0].add(q.fplan);
        joined[1].add(q.splan);
        joined[2].add(q.mplan);
    }
    for (const PlanBase *t : {&ft, &st_, &mt}) {
        for (int k = 0; k < K_NKINDS; ++k)
            if (t->kind[k] > kCodeMask) {
                error = "batch too large for one handle: more than 2^28 tasks of one kind";
                return HLU_EINVAL;
            }
        if (t->edges > INT32_MAX || t->tasks > INT32_MAX || t->terms > INT32_MAX || t->pieces > INT32_MAX) {
            error = "batch too large for one handle: more than 2^31 tasks or dependencies";
            return HLU_EINVAL;
        }
    }
    if (n_leaves + nsplit > INT32_MAX) {
        error = "batch too large for one handle: more than 2^31 blocks";
        return HLU_EINVAL;
    }
    // the shared regions at the end of the arenas
    f_ident_off = fpos;
    fpos = align8(fpos + int64_t(max_leaf) * max_leaf);
    f_solve_off = fpos;
    fpos = align8(fpos + int64_t(n) * W);
    f_z_off = -1;
    if (any_z) {
        f_z_off = fpos;
        fpos = align8(fpos + int64_t(n) * W);
    }
    f_elems = fpos;
    a_x_off = apos;
    apos = align8(apos + int64_t(n) * W);
    a_y_off = apos;
    apos = align8(apos + int64_t(n) * W);
    a_elems = apos;
    nrhs_slot = nslot;
    n_slots = nslot + 1;
    for (int32_t i = 0; i < count; ++i) {
        const Planner &q = *parts[i];
        const int32_t ni = q.n, r0 = rb[i];
        fs[i].nrhs = as[i].nrhs = nrhs_slot;
        fs[i].moved.push_back(Moved{q.f_solve_off, int64_t(ni) * W, ni, f_solve_off + r0, n});
        if (q.f_z_off >= 0) fs[i].moved.push_back(Moved{q.f_z_off, int64_t(ni) * W, ni, f_z_off + r0, n});
        fs[i].moved.push_back(Moved{q.f_ident_off, int64_t(q.max_leaf) * q.max_leaf, q.max_leaf, f_ident_off,
                                    max_leaf});
        as[i].moved.push_back(Moved{q.a_x_off, int64_t(ni) * W, ni, a_x_off + r0, n});
        as[i].moved.push_back(Moved{q.a_y_off, int64_t(ni) * W, ni, a_y_off + r0, n});
    }
    try {
        slot_init.assign(n_slots, 0);
        fstore.assign(n_leaves + nsplit, Store{});
        astore.assign(n_leaves, Store{});
        inv_cl.assign(ninv, 0);
        inv_L_off.assign(ninv, 0);
        inv_U_off.assign(ninv, 0);
        inv_index.assign(cl.size(), -1);
        fplan = Plan();
        splan = Plan();
        mplan = Plan();
        reserve_joined(fplan, ft);
        reserve_joined(splan, st_);
        reserve_joined(mplan, mt);
    } catch (const std::bad_alloc &) {
        error = "host memory exhausted while joining the plans";
        return HLU_ENOMEM;
    }
    // join in problem order: the stores and inverse blocks, then the plans' groups of arrays each on
    // its own thread, freeing what it has appended
    auto join_plans = [&](int group) {
        for (int32_t i = 0; i < count; ++i) {
            Planner &q = *parts[i];
            join_group(group, q.fplan, fb[i], fs[i], fplan);
            join_group(group, q.splan, sb[i], fs[i], splan);
            join_group(group, q.mplan, mb[i], as[i], mplan);
        }
    };
    for (int32_t i = 0; i < count; ++i) {
        Planner &q = *parts[i];
        const Shift &f = fs[i], &a = as[i];
        std::copy(q.slot_init.begin(), q.slot_init.end(), slot_init.begin() + f.slot);
        for (size_t j = 0; j < q.fstore.size(); ++j) {
            Store s = q.fstore[j];
            s.t += f.cluster;
            s.s += f.cluster;
            s.D_off = f.off(s.D_off);
            s.U_off = f.off(s.U_off);
            s.V_off = f.off(s.V_off);
            s.kslot = f.slot_of(s.kslot);
            fstore[f.store(int32_t(j))] = s;
        }
        for (int64_t j = 0; j < q.n_leaves; ++j) {
            Store s = q.astore[j];
            s.t += a.cluster;
            s.s += a.cluster;
            s.D_off = a.off(s.D_off);
            s.U_off = a.off(s.U_off);
            s.V_off = a.off(s.V_off);
            astore[a.leaf + j] = s;
        }
        for (size_t j = 0; j < q.inv_cl.size(); ++j) {
            inv_cl[inv_base[i] + j] = q.inv_cl[j] + f.cluster;
            inv_L_off[inv_base[i] + j] = f.off(q.inv_L_off[j]);
            inv_U_off[inv_base[i] + j] = f.off(q.inv_U_off[j]);
            inv_index[q.inv_cl[j] + f.cluster] = int32_t(inv_base[i] + j);
        }
    }
    run_parts(kJoinGroups, join_plans);
    for (int32_t i = 0; i < count; ++i) parts[i].reset();
    // graph-wide figures (the problems run side by side), and the roots of all problems in one
    // order of priority (longest remaining path first), as a single plan orders its own
    for (int w = 0; w < 3; ++w) {
        Plan &q = w == 0 ? fplan : w == 1 ? splan : mplan;
        const Joined &j = joined[w];
        q.n_waves = j.n_waves;
        q.critical_us = j.critical_us;
        q.max_kcap = j.max_kcap;
        q.temp_elems = j.temp_elems;
        q.temp_peak_elems = j.temp_peak_elems;
        q.scratch_base = w == 2 ? a_elems : f_elems;
        q.scratch_elems = 0;
        std::vector<int32_t> idx(q.roots.size());
        for (size_t r = 0; r < idx.size(); ++r) idx[r] = int32_t(r);
        std::stable_sort(idx.begin(), idx.end(), [&](int32_t a, int32_t b) { return q.root_bl[a] > q.root_bl[b]; });
        std::vector<int32_t> roots(idx.size());
        std::vector<float> bl(idx.size());
        for (size_t r = 0; r < idx.size(); ++r) {
            roots[r] = q.roots[idx[r]];
            bl[r] = q.root_bl[idx[r]];
        }
        q.roots.swap(roots);
        q.root_bl.swap(bl);
    }
    return HLU_OK;
}

}  // namespace hlu
