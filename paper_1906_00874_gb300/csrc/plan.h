// Host planner: expands the H-LU recursion into a task graph with dependency
// waves, and lays out the device arenas.
//
// The recursion is the 2 x 2 block LU of Sec. 3.1 at every partitioned diagonal
// block (factor the leading block, solve the two off-diagonal blocks with its
// factors, Schur update, factor the trailing block), each off-diagonal solve
// broken into block substitution as in Sec. 5.2 when that block is partitioned.
// Dependencies between tasks are found from the matrix regions they read and
// write, at the granularity of leaf clusters: every stored object (a dense
// block, the U or V factor of a low-rank block, a temporary panel) is cut into
// cells along the leaf clusters of its row (and column) cluster.  This plays
// the role of the skeleton array of Sec. 5.1 - a fixed table of representants,
// built once, that is decoupled from the storage whose sizes change during the
// factorisation - and, because all tasks of all recursion levels are analysed
// in one domain, it exposes the cross-level parallelism that weak dependencies
// and early release give in Sec. 5.2.  Tasks are grouped into waves
// (longest-path levels); the tasks of one wave are independent.
#pragma once
#include <stdint.h>

#include <array>
#include <initializer_list>
#include <string>
#include <system_error>
#include <thread>
#include <vector>

#include "tasks.h"

namespace hlu {

// Runs part(q) for q = 0 .. n - 1: part 0 on the calling thread, the others on threads of their own,
// and any part whose thread cannot be made on the calling thread too.
template <class F>
void run_parts(int n, const F &part) {
    std::vector<std::thread> pool;
    std::vector<int> here;
    pool.reserve(size_t(n > 1 ? n - 1 : 0));
    for (int q = 1; q < n; ++q) {
        try {
            pool.emplace_back(part, q);
        } catch (const std::system_error &) {
            here.push_back(q);
        }
    }
    part(0);
    for (int q : here) part(q);
    for (std::thread &th : pool) th.join();
}

struct ClusterInfo {
    int32_t begin, size, son0, son1;
    int32_t lc_first, lc_count;  // leaf clusters below, in DoF order
};

struct Obj {
    int32_t row_cl, col_cl;  // -1: not cluster-indexed (one cell in that dimension)
    int32_t nr, nc;
    int64_t cell_base;
};

struct View {
    Panel p;
    int32_t obj;
    int32_t r_cl, c_cl;  // cluster of the view's rows / columns, -1 if none
    bool trans;          // view rows run along the object's columns
};

// B_ZERO: a block between two different instances of a batch (structurally zero: no leaf, no task).
enum BKind : int32_t { B_DENSE = 0, B_LOWRANK = 1, B_PART = 2, B_ZERO = 3 };

struct Block {
    int32_t t, s;
    BKind kind;
    int32_t id;  // storage id for leaves (input leaves first, then temporary splits)
    Block *son[2][2];
};

// Storage of one leaf (or temporary split block) in one arena.
struct Store {
    int32_t kind;  // B_DENSE / B_LOWRANK
    int32_t t, s, m, n;
    int64_t D_off, U_off, V_off;
    int32_t cap;     // column capacity of U and V
    int32_t kslot;   // dynamic rank slot, -1 if static
    int32_t krank;   // static rank (A_H arena) or input rank
    int32_t objD, objU, objV;
};

struct Launch {
    int32_t wave, kind, start, count;
};

struct Plan {
    std::vector<TGetrf> getrf;
    std::vector<TTrsm> trsm;
    std::vector<TProject> project;
    std::vector<TAccum> accum;
    std::vector<TRadd> radd;
    std::vector<TSplit> split;
    std::vector<Term> terms;
    std::vector<Piece> pieces;
    std::vector<int32_t> wave[K_NKINDS];
    std::vector<Launch> launches;
    int32_t n_waves = 0;
    int64_t n_tasks = 0;
    // explicit dependency graph over all tasks, numbered in emission order
    std::vector<int32_t> task_code;           // (kind << kCodeShift) | index into the kind's (wave-sorted) array
    std::vector<int32_t> pred_ptr, pred_idx;  // predecessors (CSR), built during emission
    std::vector<int32_t> succ_ptr, succ_idx;  // successors (CSR), built by finalize
    std::vector<int32_t> indeg, roots;
    std::vector<float> root_bl;               // priority of every root (its longest path to the end, µs)
    int64_t n_edges = 0;
    int64_t scratch_base = 0, scratch_elems = 0;
    int32_t max_kcap = 0;
    double critical_us = 0.0;  // longest path of the graph under the per-kind task latencies (µs)
    // product temporaries: elements in all, and the largest sum over one dependency level of the
    // temporaries in use at that level (from their first writer's level to their last reader's)
    int64_t temp_elems = 0, temp_peak_elems = 0;
    // tasks per kind and the in-degree of the last task, kept when the task arrays are released
    int64_t kind_count[K_NKINDS] = {0, 0, 0, 0, 0, 0};
    int32_t last_indeg = 0;

    // Frees the task arrays and the graph (once they are on the device), keeping the figures above,
    // the sizes and the wave launches.
    void release_tasks();
};

struct PlanOptions {
    int32_t rank_cap = 32;
    int32_t nrhs_max = 64;
    int32_t kmax_core = 96;  // largest stacked rank a rounded addition handles (at most 128: the
                             // truncation core keeps a column of its right factor in one warp)
    bool wave_order = true;   // sort each kind's tasks by wave and list the wave launches (only the
                              // wave schedule needs them; the data-flow schedule runs any order)
    int32_t inv_block = 1024; // the largest diagonal blocks of at most this order (at least the
                             // largest leaf) are inverted after the factorisation, and the solve
                             // applies the inverses as products; 0: plain block substitution
    bool temp_reuse = false;  // the factorisation's product temporaries share device regions by
                             // dependency-level intervals (relocate_temps); false: each its own region
    int32_t batch_threads = 0;  // batch, data-flow schedule: the problems are planned on this many host
                                // threads (0: all hardware threads) and their graphs joined
                                // (plan_batch); < 0: one plan of the whole forest on one thread.
                                // Unless this is < 0, a factorisation plan that plan_all emits in
                                // one piece has its dependency analysis on a second thread (so do
                                // the problems of a batch when the pool has two threads for each).
};

class Planner {
public:
    // ---- inputs (validated copies)
    int32_t n = 0;
    std::vector<ClusterInfo> cl;
    // batch of independent H-matrices: instance of every cluster (-1 for the clusters above the
    // instances' roots); empty for a single H-matrix
    std::vector<int32_t> inst;
    int32_t n_inst = 1;
    std::vector<int32_t> perm;
    std::vector<int32_t> lc_ids;  // leaf clusters in DoF order
    int32_t max_leaf = 0;
    int64_t n_leaves = 0;
    std::vector<int32_t> leaf_row, leaf_col, leaf_rank;
    std::vector<int8_t> leaf_kind;
    std::vector<int64_t> leaf_offset;
    PlanOptions opt;

    // ---- block tree
    std::vector<Block *> blocks_owned;
    Block *root = nullptr;

    // ---- factor arena (element type chosen by the caller) and A_H arena (FP64)
    std::vector<Store> fstore;   // input leaves then temporary split blocks
    std::vector<Store> astore;   // input leaves only
    int64_t f_elems = 0, a_elems = 0;
    int64_t f_ident_off = 0;     // max_leaf x max_leaf identity in the factor arena
    int32_t n_slots = 0;         // dynamic dimension slots
    std::vector<int32_t> slot_init;  // initial value of every slot
    int32_t nrhs_slot = -1;      // solve / matvec panel width
    int64_t f_solve_off = 0;     // n x nrhs_max panel (factor arena)
    int64_t a_x_off = 0, a_y_off = 0;  // n x nrhs_max panels (A_H arena)
    int64_t f_z_off = -1;        // second n x nrhs_max solve panel (inverse-block solve only)
    // inverse blocks: the diagonal blocks (c, c) whose inverses L_cc^{-1}, U_cc^{-1} (dense,
    // n_c x n_c, column-major) the factorisation forms for the solve
    std::vector<int32_t> inv_cl, inv_index;  // clusters; per cluster its inverse block or -1
    std::vector<int64_t> inv_L_off, inv_U_off;

    Plan fplan, splan, mplan;    // factorisation, solve, matvec

    std::string error;

    ~Planner();
    // Returns 0 or an HLU_* status with `error` set.
    int build(int32_t n, int32_t n_clusters, const int32_t *perm, const int32_t *begin,
              const int32_t *size, const int32_t *son0, const int32_t *son1, int64_t n_leaves,
              const int32_t *row_cl, const int32_t *col_cl, const int8_t *kind,
              const int32_t *rank, const int64_t *offset, const double *data,
              int64_t data_len, const PlanOptions &o, const int32_t *inst = nullptr, int32_t n_inst = 0);
    // Lays out the arenas and emits the factorisation, solve and matvec plans.
    int plan_all();

    // Frees the emission state (cells, objects, block tree, predecessor lists) once the plans are made.
    void release_work();

private:
    bool batch_deferred = false;  // a batch whose problems plan_all plans separately (plan_batch)
    int plan_batch();
    bool batch_layout(std::vector<int32_t> &cb, std::vector<int32_t> &ce, std::vector<int64_t> &lb,
                      std::vector<int32_t> &rb) const;

    // current plan being emitted
    Plan *P = nullptr;
    bool use_astore = false;
    bool split_accum = false;  // solve plan: split each ACCUM into its early and its latest terms
    int64_t *arena = nullptr;  // bump pointer of the current arena
    std::vector<Obj> objs;
    // per cell: the wave of its last writer, the latest wave that read it since, the last writer
    // task, and the readers since (head of a singly linked list in a pool); one record per cell so
    // that the dependency analysis touches one cache line per cell
    struct CellState {
        int32_t write_wave, read_wave, writer, rhead;
    };
    // The state of the dependency analysis (owned by the analysing thread while the emission is piped)
    struct Deps {
        std::vector<CellState> cell;
        std::vector<int32_t> pred_mark;  // per task: the last task that listed it as a predecessor
        std::vector<int32_t> rpool_task, rpool_next;
        // the tasks that touch each cell of each temporary (object, cell within the object, task, written)
        std::vector<int32_t> touch_obj, touch_cell, touch_task;
        std::vector<uint8_t> touch_write;
        // per temporary object: the first and last dependency level of a task that touches it
        std::vector<int32_t> temp_first, temp_last;
        void swap(Deps &o) {
            cell.swap(o.cell);
            pred_mark.swap(o.pred_mark);
            rpool_task.swap(o.rpool_task);
            rpool_next.swap(o.rpool_next);
            touch_obj.swap(o.touch_obj);
            touch_cell.swap(o.touch_cell);
            touch_task.swap(o.touch_task);
            touch_write.swap(o.touch_write);
            temp_first.swap(o.temp_first);
            temp_last.swap(o.temp_last);
        }
    };
    Deps dep;
    int32_t ident_obj = -1;
    bool no_flops = false;  // emitted tasks are not counted in the model flops
    std::vector<int32_t> inv_objL, inv_objU;

    int32_t new_obj(int32_t row_cl, int32_t col_cl, int32_t nr_if_none = 1);
    int32_t new_slot(int32_t init);
    // owner_cl: a cluster of the problem (of a batch) the temporary belongs to
    View new_temp(int32_t row_cl, int32_t rows, int32_t cols, int32_t rslot, int32_t cslot, int32_t owner_cl);
    // Allocations of the current plan in the arena, in bump order (temp_obj >= 0: a product
    // temporary).
    struct PlanItem {
        int64_t off, size;
        int32_t temp_obj;
    };
    std::vector<PlanItem> plan_items;
    int64_t plan_begin = 0;
    std::vector<std::array<int32_t, 4>> temp_shape;  // per temporary object: problem, row cluster, rows, cols
    int64_t plan_alloc(int64_t elems, int32_t temp_obj);
    // per object: its elements when it is a temporary of the current plan (else 0)
    std::vector<int64_t> temp_size;
    void temp_levels(Plan &p) const;
    void relocate_temps(Plan &p);
    // Host threads for a piece of planning work that splits into at most `limit` parts: up to eight,
    // one when opt.batch_threads < 0.
    int host_parts(int64_t limit) const;
    void note_temp(int32_t obj, int64_t elems, const std::array<int32_t, 4> &shape);
    void cells_of(const View &v, std::vector<int64_t> &out) const;
    // The cells a view covers: rows r0..r1-1 and columns c0..c1-1 of the cell grid of an object whose
    // cells start at base with nc per row; temp_obj is the object when it is a temporary of the
    // current plan, else -1.
    struct ViewRec {
        int64_t base;
        int32_t nc, r0, r1, c0, c1, temp_obj;
    };
    void describe(const View &v, ViewRec &r) const;
    // The dependency analysis of task g (reads first, then writes): its predecessors, its wave, the
    // level interval of the temporaries it touches.  Returns the wave.
    int32_t analyze(Deps &d, std::vector<int32_t> &pred_ptr, std::vector<int32_t> &pred_idx, const ViewRec *v,
                    size_t nr, size_t nw, int32_t g) const;
    // Factorisation emission with the analysis on a second host thread: emit_views hands the
    // tasks' cells to it in chunks (pipe_begin / pipe_end around the recursion).
    struct Pipe;
    Pipe *pipe = nullptr;
    bool pipe_begin();  // false (nothing started) when no thread can be made
    void reserve_factorisation();
    int pipe_end();
    int32_t emit_views(Kind k, const View *const *reads, size_t nr, const View *const *writes, size_t nw);
    int32_t emit(Kind k, std::initializer_list<const View *> reads, std::initializer_list<const View *> writes) {
        return emit_views(k, reads.begin(), reads.size(), writes.begin(), writes.size());
    }
    int32_t emit(Kind k, const std::vector<const View *> &reads, std::initializer_list<const View *> writes) {
        return emit_views(k, reads.data(), reads.size(), writes.begin(), writes.size());
    }

    Store &st(const Block *b) { return use_astore ? astore[b->id] : fstore[b->id]; }
    View viewD(const Block *b);
    View viewU(const Block *b);
    View viewV(const Block *b);
    View ident(int32_t c);
    View rows(const View &v, int32_t sub) const;
    static View transpose(const View &v);

    void collect_leaves(Block *b, std::vector<Block *> &out);

    // the recursion
    void lu(Block *b);
    void trsm_l(Block *L, Block *X);
    void trsm_u(Block *U, Block *X);
    void trsm_l_panel(Block *L, const View &P);
    void trsm_u_panel(Block *U, const View &P);
    void hmm(const View &out, double alpha, bool overwrite, Block *M, bool trans, const View &X,
             int32_t wdst = -1, int32_t wsrc = -1);
    struct Prod { View U, V; };
    Prod product(Block *A, Block *B);
    void add_into(Block *C, double alpha, const Prod &p);
    void addmul(Block *C, double alpha, Block *A, Block *B);
    void radd(Block *C, bool include_self, const std::vector<Piece> &pcs, const std::vector<View> &pviews);
    void solve_lower(Block *F, const View &Y);
    void solve_upper(Block *F, const View &Y);
    // inverse-block solve
    bool leaf_is_dense(int32_t q, int32_t j) const;
    void choose_inverses(int32_t t, int32_t bound);
    void plan_inverses();
    void inv_solve_lower(Block *F, const View &Y, int32_t s0);
    void inv_solve_upper(Block *F, const View &Y, int32_t e0);
    void apply_inverse(int32_t idx, bool upper, const View &in, const View &out);
    void solve_lower_pp(Block *F, const View &Y, const View &Z);
    void solve_upper_pp(Block *F, const View &Z, const View &Y);

    int build_tree();
    void layout_factor_arena();
    void layout_a_arena();
    void finalize_alloc(Plan &p, int64_t *bump) const;
    void finalize_graph(Plan &p) const;
    void begin_plan(Plan &p, bool astore_mode, int64_t *bump);
};

}  // namespace hlu
