// CPU executor of the planner's task lists (test infrastructure, not part of the library).
//
// The host planner (paper_1906_00874_gb300/csrc/plan.cpp) expands the H-LU recursion of Sec. 3.1
// into tasks of six kinds with explicit dependencies.  This file runs those tasks on the CPU in
// double precision, in a random order that respects the dependencies (or in wave order), so that the
// task lists themselves can be checked against the oracle without a GPU: wrong operands, a missing
// or superfluous dependency, or a wrong truncation point show up as a different factorisation.
//
// The rounded addition is computed here by its plain definition (stack the factors, Householder QR of
// both stacks, pivoted QR of the core stopped at 1e-13 of the first pivot, one-sided Jacobi SVD,
// keep sigma > eps sigma_1), the same T_eps as the library's kernels and the oracle.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <random>
#include <vector>

#include "plan.h"

using namespace hlu;

namespace {

struct Exec {
    std::vector<double> A;  // the factor arena, double precision
    std::vector<int32_t> kd;  // dynamic dimensions
    double eps = 0.0;
    int err = 0;

    int rows(const Panel &p) const { return p.rslot >= 0 ? kd[p.rslot] : p.rows; }
    int cols(const Panel &p) const { return p.cslot >= 0 ? kd[p.cslot] : p.cols; }
    double &at(const Panel &p, int i, int j) { return A[p.off + int64_t(i) * p.rs + int64_t(j) * p.cs]; }

    void getrf(const TGetrf &t) {
        double *a = &A[t.off];
        const int m = t.m;
        for (int k = 0; k < m; ++k) {
            const double piv = a[k + k * m];
            if (!(piv != 0.0) || !std::isfinite(piv)) err = 1;
            for (int i = k + 1; i < m; ++i) a[i + k * m] /= piv;
            for (int j = k + 1; j < m; ++j)
                for (int i = k + 1; i < m; ++i) a[i + j * m] -= a[i + k * m] * a[k + j * m];
        }
    }

    void trsm(const TTrsm &t) {
        const double *L = &A[t.L_off];
        const int m = t.m, p = cols(t.P), mode = t.mode & 0xff;
        for (int c = 0; c < p; ++c) {
            if (mode == TR_LOWER_UNIT) {
                for (int i = 0; i < m; ++i) {
                    double s = at(t.P, i, c);
                    for (int l = 0; l < i; ++l) s -= L[i + l * m] * at(t.P, l, c);
                    at(t.P, i, c) = s;
                }
            } else if (mode == TR_UPPER_TRANS) {  // P := U^{-T} P
                for (int i = 0; i < m; ++i) {
                    double s = at(t.P, i, c);
                    for (int l = 0; l < i; ++l) s -= L[l + i * m] * at(t.P, l, c);
                    at(t.P, i, c) = s / L[i + i * m];
                }
            } else {  // P := U^{-1} P
                for (int i = m - 1; i >= 0; --i) {
                    double s = at(t.P, i, c);
                    for (int l = i + 1; l < m; ++l) s -= L[i + l * m] * at(t.P, l, c);
                    at(t.P, i, c) = s / L[i + i * m];
                }
            }
        }
    }

    void project(const TProject &t) {
        const int len = rows(t.F), k = cols(t.F), p = cols(t.X);
        if (t.dst0 >= 0) kd[t.dst0] = kd[t.src0];
        if (t.dst1 >= 0) kd[t.dst1] = kd[t.src1];
        for (int a = 0; a < k; ++a)
            for (int b = 0; b < p; ++b) {
                double s = 0.0;
                for (int r = 0; r < len; ++r) s += at(t.F, r, a) * at(t.X, r, b);
                at(t.T, a, b) = s;
            }
    }

    void accum(const TAccum &t, const std::vector<Term> &terms) {
        if (t.dst >= 0) kd[t.dst] = kd[t.src];
        const int m = rows(t.out), p = cols(t.out);
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < p; ++j) {
                double s = 0.0;
                for (int q = 0; q < t.nterms; ++q) {
                    const Term &tm = terms[t.term0 + q];
                    const int in = cols(tm.A);
                    for (int l = 0; l < in; ++l) s += at(tm.A, i, l) * at(tm.X, l, j);
                }
                at(t.out, i, j) = (t.overwrite ? 0.0 : at(t.out, i, j)) + t.alpha * s;
            }
    }

    void split(const TSplit &t) {
        const int k = kd[t.src_kslot];
        kd[t.dst_kslot] = k;
        for (int j = 0; j < k; ++j) {
            for (int i = 0; i < t.mu; ++i) A[t.dstU + i + int64_t(j) * t.mu] = at(t.srcU, i, j);
            for (int i = 0; i < t.nv; ++i) A[t.dstV + i + int64_t(j) * t.nv] = at(t.srcV, i, j);
        }
    }

    // Householder QR in place (W: m x K, ld m): reflector j below the diagonal (v_j[j] = 1), R above.
    static void householder(double *W, int m, int K, std::vector<double> &tau) {
        const int kk = std::min(m, K);
        tau.assign(kk, 0.0);
        for (int j = 0; j < kk; ++j) {
            double *x = W + int64_t(j) * m;
            double nrm = 0.0;
            for (int i = j; i < m; ++i) nrm += x[i] * x[i];
            nrm = std::sqrt(nrm);
            if (nrm == 0.0) continue;
            const double alpha = x[j] >= 0.0 ? -nrm : nrm, v0 = x[j] - alpha;
            for (int i = j + 1; i < m; ++i) x[i] /= v0;
            tau[j] = (alpha - x[j]) / alpha;
            x[j] = alpha;
            for (int c = j + 1; c < K; ++c) {
                double *y = W + int64_t(c) * m, s = y[j];
                for (int i = j + 1; i < m; ++i) s += x[i] * y[i];
                s *= tau[j];
                y[j] -= s;
                for (int i = j + 1; i < m; ++i) y[i] -= s * x[i];
            }
        }
    }

    // Z (m x nc, ld ldz) := Q Z with Q from householder().
    static void apply_q(const double *W, int m, int kk, const std::vector<double> &tau, double *Z, int ldz, int nc) {
        for (int j = kk - 1; j >= 0; --j) {
            const double *x = W + int64_t(j) * m;
            for (int c = 0; c < nc; ++c) {
                double *y = Z + int64_t(c) * ldz, s = y[j];
                for (int i = j + 1; i < m; ++i) s += x[i] * y[i];
                s *= tau[j];
                y[j] -= s;
                for (int i = j + 1; i < m; ++i) y[i] -= s * x[i];
            }
        }
    }

    // One-sided Jacobi on the columns of B (r x c) with the rotations accumulated in J (c x c).
    static void jacobi(std::vector<double> &B, int r, int c, std::vector<double> &J) {
        J.assign(size_t(c) * c, 0.0);
        for (int i = 0; i < c; ++i) J[i + i * c] = 1.0;
        const double tol = 4.0 * r * 2.220446049250313e-16;
        for (int sweep = 0; sweep < 30; ++sweep) {
            bool rotated = false;
            for (int p = 0; p < c - 1; ++p)
                for (int q = p + 1; q < c; ++q) {
                    double a = 0.0, b = 0.0, g = 0.0;
                    for (int i = 0; i < r; ++i) {
                        a += B[i + p * r] * B[i + p * r];
                        b += B[i + q * r] * B[i + q * r];
                        g += B[i + p * r] * B[i + q * r];
                    }
                    if (g == 0.0 || std::fabs(g) <= tol * std::sqrt(a * b)) continue;
                    rotated = true;
                    const double zeta = (b - a) / (2.0 * g);
                    const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
                    const double cs = 1.0 / std::sqrt(1.0 + t * t), sn = cs * t;
                    for (int i = 0; i < r; ++i) {
                        const double x = B[i + p * r], y = B[i + q * r];
                        B[i + p * r] = cs * x - sn * y;
                        B[i + q * r] = sn * x + cs * y;
                    }
                    for (int i = 0; i < c; ++i) {
                        const double x = J[i + p * c], y = J[i + q * c];
                        J[i + p * c] = cs * x - sn * y;
                        J[i + q * c] = sn * x + cs * y;
                    }
                }
            if (!rotated) break;
        }
    }

    void radd(const TRadd &t, const std::vector<Piece> &pieces) {
        const int m = t.m, n = t.n;
        int K = t.include_self ? kd[t.kslot] : 0;
        for (int q = 0; q < t.npieces; ++q) K += cols(pieces[t.piece0 + q].U);
        std::vector<double> WU(size_t(m) * std::max(K, 1), 0.0), WV(size_t(n) * std::max(K, 1), 0.0);
        int col = 0;
        if (t.include_self)
            for (int j = 0; j < kd[t.kslot]; ++j, ++col) {
                for (int i = 0; i < m; ++i) WU[i + size_t(col) * m] = A[t.U_off + i + int64_t(j) * m];
                for (int i = 0; i < n; ++i) WV[i + size_t(col) * n] = A[t.V_off + i + int64_t(j) * n];
            }
        for (int q = 0; q < t.npieces; ++q) {
            const Piece &pc = pieces[t.piece0 + q];
            const int k = cols(pc.U), mu = rows(pc.U), nv = rows(pc.V);
            for (int j = 0; j < k; ++j, ++col) {
                for (int i = 0; i < mu; ++i) WU[pc.roff + i + size_t(col) * m] = pc.coef * at(pc.U, i, j);
                for (int i = 0; i < nv; ++i) WV[pc.coff + i + size_t(col) * n] = at(pc.V, i, j);
            }
        }
        if (K == 0) {
            kd[t.kslot] = 0;
            return;
        }
        std::vector<double> tu, tv;
        householder(WU.data(), m, K, tu);
        householder(WV.data(), n, K, tv);
        const int ku = std::min(m, K), kv = std::min(n, K);
        std::vector<double> M(size_t(ku) * kv, 0.0);  // core R_u R_v^T
        for (int i = 0; i < ku; ++i)
            for (int j = 0; j < kv; ++j) {
                double s = 0.0;
                for (int l = std::max(i, j); l < K; ++l) s += WU[i + size_t(l) * m] * WV[j + size_t(l) * n];
                M[i + size_t(j) * ku] = s;
            }
        // pivoted QR of the core, stopped at 1e-13 times the first pivot: M P = Q_M [R'; ~0]
        std::vector<int> perm(kv);
        std::vector<double> cn(kv), tq;
        for (int j = 0; j < kv; ++j) {
            perm[j] = j;
            double s = 0.0;
            for (int i = 0; i < ku; ++i) s += M[i + size_t(j) * ku] * M[i + size_t(j) * ku];
            cn[j] = s;
        }
        int r = 0;
        double n0 = 0.0;
        for (int j = 0; j < std::min(ku, kv); ++j) {
            int p = j;
            for (int c = j + 1; c < kv; ++c)
                if (cn[c] > cn[p]) p = c;
            if (j == 0) n0 = cn[p];
            if (!(cn[p] > 1e-26 * n0)) break;
            if (p != j) {
                for (int i = 0; i < ku; ++i) std::swap(M[i + size_t(j) * ku], M[i + size_t(p) * ku]);
                std::swap(cn[j], cn[p]);
                std::swap(perm[j], perm[p]);
            }
            double *x = &M[size_t(j) * ku], nrm = 0.0;
            for (int i = j; i < ku; ++i) nrm += x[i] * x[i];
            nrm = std::sqrt(nrm);
            double tau = 0.0;
            if (nrm > 0.0) {
                const double alpha = x[j] >= 0.0 ? -nrm : nrm, v0 = x[j] - alpha;
                for (int i = j + 1; i < ku; ++i) x[i] /= v0;
                tau = (alpha - x[j]) / alpha;
                x[j] = alpha;
            }
            tq.push_back(tau);
            for (int c = j + 1; c < kv; ++c) {
                double *y = &M[size_t(c) * ku], s = y[j];
                for (int i = j + 1; i < ku; ++i) s += x[i] * y[i];
                s *= tau;
                y[j] -= s;
                double t2 = 0.0;
                for (int i = j + 1; i < ku; ++i) {
                    y[i] -= s * x[i];
                    t2 += y[i] * y[i];
                }
                cn[c] = t2;
            }
            r = j + 1;
        }
        // SVD of R'^T (kv x r) by one-sided Jacobi: R'^T J = C, sigma_j = |C_j|
        std::vector<double> Cm(size_t(kv) * std::max(r, 1), 0.0), J;
        for (int i = 0; i < r; ++i)
            for (int c = i; c < kv; ++c) Cm[c + size_t(i) * kv] = M[i + size_t(c) * ku];
        jacobi(Cm, kv, r, J);
        std::vector<std::pair<double, int>> sg(std::max(r, 1));
        for (int j = 0; j < r; ++j) {
            double s = 0.0;
            for (int i = 0; i < kv; ++i) s += Cm[i + size_t(j) * kv] * Cm[i + size_t(j) * kv];
            sg[j] = {-std::sqrt(s), j};
        }
        std::sort(sg.begin(), sg.begin() + r);
        const double s1 = r ? -sg[0].first : 0.0;
        int k = 0;
        if (s1 > 0.0)
            for (int j = 0; j < r; ++j) k += -sg[j].first > eps * s1;
        if (k > t.cap) {
            err = 2;
            k = t.cap;
        }
        // U = Q_u [Q_M [J_sel Sigma; 0]; 0], V = Q_v [P C_sel Sigma^{-1}; 0]
        std::vector<double> Z(size_t(m) * std::max(k, 1), 0.0), Y(size_t(n) * std::max(k, 1), 0.0);
        for (int c = 0; c < k; ++c) {
            const int j = sg[c].second;
            const double sig = -sg[c].first;
            for (int i = 0; i < r; ++i) Z[i + size_t(c) * m] = J[i + size_t(j) * r] * sig;
        }
        for (int jj = r - 1; jj >= 0; --jj) {
            const double *x = &M[size_t(jj) * ku];
            for (int c = 0; c < k; ++c) {
                double *y = &Z[size_t(c) * m], s = y[jj];
                for (int i = jj + 1; i < ku; ++i) s += x[i] * y[i];
                s *= tq[jj];
                y[jj] -= s;
                for (int i = jj + 1; i < ku; ++i) y[i] -= s * x[i];
            }
        }
        for (int c = 0; c < k; ++c) {
            const int j = sg[c].second;
            const double sig = -sg[c].first;
            for (int i = 0; i < kv; ++i) Y[perm[i] + size_t(c) * n] = Cm[i + size_t(j) * kv] / sig;
        }
        apply_q(WU.data(), m, ku, tu, Z.data(), m, k);
        apply_q(WV.data(), n, kv, tv, Y.data(), n, k);
        for (int c = 0; c < k; ++c) {
            for (int i = 0; i < m; ++i) A[t.U_off + i + int64_t(c) * m] = Z[i + size_t(c) * m];
            for (int i = 0; i < n; ++i) A[t.V_off + i + int64_t(c) * n] = Y[i + size_t(c) * n];
        }
        kd[t.kslot] = k;
    }

    void run_task(const Plan &p, int g) {
        const int code = p.task_code[g], kind = code >> kCodeShift, i = code & kCodeMask;
        switch (kind) {
            case K_GETRF: getrf(p.getrf[i]); break;
            case K_TRSM: trsm(p.trsm[i]); break;
            case K_PROJECT: project(p.project[i]); break;
            case K_ACCUM: accum(p.accum[i], p.terms); break;
            case K_RADD: radd(p.radd[i], p.pieces); break;
            default: split(p.split[i]); break;
        }
    }

    // Every task once, in a random order that respects the dependencies; returns the count run.
    int64_t run(const Plan &p, uint64_t seed) {
        std::mt19937_64 rng(seed);
        std::vector<int32_t> indeg = p.indeg, ready(p.roots.begin(), p.roots.end());
        int64_t done = 0;
        while (!ready.empty()) {
            const size_t j = rng() % ready.size();
            const int g = ready[j];
            ready[j] = ready.back();
            ready.pop_back();
            run_task(p, g);
            ++done;
            for (int e = p.succ_ptr[g]; e < p.succ_ptr[g + 1]; ++e)
                if (--indeg[p.succ_idx[e]] == 0) ready.push_back(p.succ_idx[e]);
        }
        return done;
    }
};

}  // namespace

// Plans the H-matrix, runs the factorisation's tasks and then one solve pass on b (n x nrhs,
// cluster order, overwritten by x), and returns the factors in the input leaf layout.  With inst
// (the problem of every cluster, -1 above the problems), the H-matrix is a batch of n_inst problems
// with one tolerance eps, planned per problem on batch_threads threads and joined (plan_batch; 0:
// all hardware threads) or, with batch_threads < 0, as one forest.  temp_reuse != 0: the product
// temporaries share regions (relocate_temps).
// Status: 0, the planner's status, or -1 (not every task ran: a dependency cycle) / -2 (a task
// failed: zero pivot or rank capacity).
extern "C" int plan_execute(int32_t n, int32_t n_clusters, const int32_t *perm, const int32_t *begin,
                            const int32_t *size, const int32_t *son0, const int32_t *son1, int64_t n_leaves,
                            const int32_t *row_cl, const int32_t *col_cl, const int8_t *kind, const int32_t *rank,
                            const int64_t *offset, const double *data, int64_t data_len, double eps,
                            int32_t inv_block, uint64_t seed, double *out, int64_t *out_off, int32_t *out_rank,
                            double *b, int32_t nrhs, const int32_t *inst, int32_t n_inst, int32_t temp_reuse,
                            int32_t batch_threads) {
    Planner pl;
    PlanOptions o;
    o.batch_threads = batch_threads;  // batch: < 0 one plan of the forest, else per problem and joined
    if (inv_block != 0) o.inv_block = inv_block < 0 ? 0 : inv_block;  // 0: the default, < 0: off
    o.temp_reuse = temp_reuse != 0;  // temporaries sharing regions by dependency-level intervals
    o.wave_order = false;
    int st = pl.build(n, n_clusters, perm, begin, size, son0, son1, n_leaves, row_cl, col_cl, kind, rank, offset,
                      data, data_len, o, inst, n_inst);
    if (st == 0) st = pl.plan_all();
    if (st) return st;
    Exec ex;
    ex.eps = eps;
    ex.A.assign(size_t(pl.f_elems), 0.0);
    ex.kd = pl.slot_init;
    for (int64_t l = 0; l < n_leaves; ++l) {
        const Store &s = pl.fstore[l];
        if (s.kind == B_DENSE) {
            std::copy(data + offset[l], data + offset[l] + int64_t(s.m) * s.n, ex.A.begin() + s.D_off);
        } else {
            const int k = rank[l];
            std::copy(data + offset[l], data + offset[l] + int64_t(s.m) * k, ex.A.begin() + s.U_off);
            std::copy(data + offset[l] + int64_t(s.m) * k, data + offset[l] + int64_t(s.m + s.n) * k,
                      ex.A.begin() + s.V_off);
        }
    }
    for (int i = 0; i < pl.max_leaf; ++i) ex.A[pl.f_ident_off + i + int64_t(i) * pl.max_leaf] = 1.0;
    if (ex.run(pl.fplan, seed) != pl.fplan.n_tasks) return -1;
    if (ex.err) return -2;
    int64_t pos = 0;
    for (int64_t l = 0; l < n_leaves; ++l) {
        const Store &s = pl.fstore[l];
        out_off[l] = pos;
        if (s.kind == B_DENSE) {
            for (int64_t i = 0; i < int64_t(s.m) * s.n; ++i) out[pos++] = ex.A[s.D_off + i];
            out_rank[l] = 0;
        } else {
            const int k = ex.kd[s.kslot];
            out_rank[l] = k;
            for (int64_t i = 0; i < int64_t(s.m) * k; ++i) out[pos++] = ex.A[s.U_off + i];
            for (int64_t i = 0; i < int64_t(s.n) * k; ++i) out[pos++] = ex.A[s.V_off + i];
        }
    }
    ex.kd[pl.nrhs_slot] = nrhs;
    for (int j = 0; j < nrhs; ++j)
        for (int i = 0; i < n; ++i) ex.A[pl.f_solve_off + i + int64_t(j) * n] = b[i + int64_t(j) * n];
    if (ex.run(pl.splan, seed + 1) != pl.splan.n_tasks) return -1;
    for (int j = 0; j < nrhs; ++j)
        for (int i = 0; i < n; ++i) b[i + int64_t(j) * n] = ex.A[pl.f_solve_off + i + int64_t(j) * n];
    return ex.err ? -2 : 0;
}

namespace {

bool same(const Panel &a, const Panel &b) {
    return a.off == b.off && a.rows == b.rows && a.cols == b.cols && a.rslot == b.rslot && a.cslot == b.cslot &&
           a.rs == b.rs && a.cs == b.cs;
}

// Every field of every task descriptor, term and piece of two plans.
bool same_descriptors(const Plan &x, const Plan &y) {
    if (x.getrf.size() != y.getrf.size() || x.trsm.size() != y.trsm.size() || x.project.size() != y.project.size() ||
        x.accum.size() != y.accum.size() || x.radd.size() != y.radd.size() || x.split.size() != y.split.size() ||
        x.terms.size() != y.terms.size() || x.pieces.size() != y.pieces.size())
        return false;
    for (size_t i = 0; i < x.getrf.size(); ++i) {
        const TGetrf &a = x.getrf[i], &b = y.getrf[i];
        if (a.off != b.off || a.m != b.m || a.leaf != b.leaf) return false;
    }
    for (size_t i = 0; i < x.trsm.size(); ++i) {
        const TTrsm &a = x.trsm[i], &b = y.trsm[i];
        if (a.L_off != b.L_off || a.m != b.m || a.mode != b.mode || !same(a.P, b.P)) return false;
    }
    for (size_t i = 0; i < x.project.size(); ++i) {
        const TProject &a = x.project[i], &b = y.project[i];
        if (!same(a.F, b.F) || !same(a.X, b.X) || !same(a.T, b.T) || a.dst0 != b.dst0 || a.src0 != b.src0 ||
            a.dst1 != b.dst1 || a.src1 != b.src1 || a.no_flops != b.no_flops)
            return false;
    }
    for (size_t i = 0; i < x.accum.size(); ++i) {
        const TAccum &a = x.accum[i], &b = y.accum[i];
        if (!same(a.out, b.out) || a.alpha != b.alpha || a.overwrite != b.overwrite || a.term0 != b.term0 ||
            a.nterms != b.nterms || a.dst != b.dst || a.src != b.src || a.credit != b.credit)
            return false;
    }
    for (size_t i = 0; i < x.terms.size(); ++i)
        if (!same(x.terms[i].A, y.terms[i].A) || !same(x.terms[i].X, y.terms[i].X)) return false;
    for (size_t i = 0; i < x.radd.size(); ++i) {
        const TRadd &a = x.radd[i], &b = y.radd[i];
        if (a.U_off != b.U_off || a.V_off != b.V_off || a.scratch_off != b.scratch_off || a.m != b.m || a.n != b.n ||
            a.cap != b.cap || a.kslot != b.kslot || a.include_self != b.include_self || a.piece0 != b.piece0 ||
            a.npieces != b.npieces || a.Kcap != b.Kcap || a.target != b.target || a.inst != b.inst)
            return false;
    }
    for (size_t i = 0; i < x.pieces.size(); ++i) {
        const Piece &a = x.pieces[i], &b = y.pieces[i];
        if (a.coef != b.coef || !same(a.U, b.U) || !same(a.V, b.V) || a.roff != b.roff || a.coff != b.coff)
            return false;
    }
    for (size_t i = 0; i < x.split.size(); ++i) {
        const TSplit &a = x.split[i], &b = y.split[i];
        if (!same(a.srcU, b.srcU) || !same(a.srcV, b.srcV) || a.dstU != b.dstU || a.dstV != b.dstV || a.mu != b.mu ||
            a.nv != b.nv || a.src_kslot != b.src_kslot || a.dst_kslot != b.dst_kslot)
            return false;
    }
    return true;
}

}  // namespace

// Plans the H-matrix twice, with the factorisation's dependency analysis on a second thread
// (batch_threads = 0) and all on one thread (batch_threads = -1), and compares the three plans:
// every task descriptor, term and piece, task codes, waves, predecessor and successor lists,
// in-degrees, roots and their priorities, the dynamic-size slots, the leaves' stores and the
// arena layout.  Returns 0 when they are equal, else 1 + the index of the first array that differs
// (plan * 16 + array), or the planner's status.
extern "C" int plan_graphs_equal(int32_t n, int32_t n_clusters, const int32_t *perm, const int32_t *begin,
                                 const int32_t *size, const int32_t *son0, const int32_t *son1, int64_t n_leaves,
                                 const int32_t *row_cl, const int32_t *col_cl, const int8_t *kind,
                                 const int32_t *rank, const int64_t *offset, const double *data, int64_t data_len,
                                 int32_t inv_block, int32_t temp_reuse) {
    Planner pl[2];
    for (int v = 0; v < 2; ++v) {
        PlanOptions o;
        o.batch_threads = v == 0 ? 0 : -1;
        if (inv_block != 0) o.inv_block = inv_block < 0 ? 0 : inv_block;
        o.temp_reuse = temp_reuse != 0;
        o.wave_order = false;
        int st = pl[v].build(n, n_clusters, perm, begin, size, son0, son1, n_leaves, row_cl, col_cl, kind, rank,
                             offset, data, data_len, o);
        if (st == 0) st = pl[v].plan_all();
        if (st) return st;
    }
    if (pl[0].f_elems != pl[1].f_elems || pl[0].a_elems != pl[1].a_elems || pl[0].f_solve_off != pl[1].f_solve_off ||
        pl[0].f_z_off != pl[1].f_z_off || pl[0].a_x_off != pl[1].a_x_off || pl[0].a_y_off != pl[1].a_y_off ||
        pl[0].slot_init != pl[1].slot_init || pl[0].nrhs_slot != pl[1].nrhs_slot ||
        pl[0].inv_L_off != pl[1].inv_L_off || pl[0].inv_U_off != pl[1].inv_U_off)
        return 1;
    for (int64_t l = 0; l < n_leaves; ++l) {
        const Store &a = pl[0].fstore[l], &b = pl[1].fstore[l];
        if (a.D_off != b.D_off || a.U_off != b.U_off || a.V_off != b.V_off || a.kslot != b.kslot || a.cap != b.cap)
            return 1;
    }
    const Plan *a[3] = {&pl[0].fplan, &pl[0].splan, &pl[0].mplan}, *b[3] = {&pl[1].fplan, &pl[1].splan, &pl[1].mplan};
    for (int q = 0; q < 3; ++q) {
        const Plan &x = *a[q], &y = *b[q];
        const int code = 2 + 16 * q;
        if (x.n_tasks != y.n_tasks || x.n_waves != y.n_waves || x.n_edges != y.n_edges) return code;
        if (x.temp_elems != y.temp_elems || x.temp_peak_elems != y.temp_peak_elems) return code + 1;
        if (x.task_code != y.task_code) return code + 2;
        for (int k = 0; k < K_NKINDS; ++k)
            if (x.wave[k] != y.wave[k]) return code + 3;
        if (x.pred_ptr != y.pred_ptr || x.pred_idx != y.pred_idx) return code + 4;
        if (x.succ_ptr != y.succ_ptr || x.succ_idx != y.succ_idx) return code + 5;
        if (x.indeg != y.indeg || x.roots != y.roots || x.root_bl != y.root_bl) return code + 6;
        if (x.critical_us != y.critical_us) return code + 7;
        if (!same_descriptors(x, y)) return code + 8;
    }
    return 0;
}
