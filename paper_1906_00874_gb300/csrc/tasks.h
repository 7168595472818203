// Task descriptors shared by the host planner and the device kernels.
//
// The H-LU recursion of Sec. 3.1 (the 2 x 2 block LU at every partitioned
// diagonal block, with the low-rank operations of the "Low-rank blocks"
// paragraph) is expanded on the host into tasks of six kinds.  Every matrix operand is a strided view ("Panel") into one device
// arena; dimensions that depend on ranks computed at run time are read from a
// device array of dynamic dimensions (kdyn) through slot indices.
#pragma once
#include <stdint.h>

namespace hlu {

// Strided view of the arena: element (i, j) is at arena[off + i*rs + j*cs].
// rows/cols are the static sizes; a slot >= 0 replaces them by kdyn[slot].
struct Panel {
    int64_t off;
    int32_t rows, cols;
    int32_t rslot, cslot;
    int32_t rs, cs;
};

// Largest leaf cluster (rows of a dense diagonal leaf) the kernels handle.
constexpr int32_t kMaxLeafRows = 128;

enum Kind : int32_t {
    K_GETRF = 0,    // unpivoted LU of a dense diagonal leaf (Sec. 3.1 "Dense blocks")
    K_TRSM = 1,     // triangular solve of a panel with a dense diagonal leaf (Sec. 3.1)
    K_PROJECT = 2,  // T = F^T X: first half of a low-rank leaf times a panel, y = U (V^T z)
    K_ACCUM = 3,    // out[seg] (+)= alpha * sum_j A_j X_j over the leaves that cover seg
    K_RADD = 4,     // rounded addition: stack factors, QR, SVD of the core, truncate
    K_SPLIT = 5,    // restriction of a low-rank block's factors to a 2x2 son
    K_NKINDS = 6
};

// A task of the data-flow graph is coded as (kind << kCodeShift) | index.
constexpr int kCodeShift = 28;
constexpr int32_t kCodeMask = (1 << kCodeShift) - 1;

enum TrsmMode : int32_t {
    TR_LOWER_UNIT = 0,   // P := L^{-1} P, L unit lower (strict lower part of the leaf)
    TR_UPPER_TRANS = 1,  // P := U^{-T} P, U upper part of the leaf (X U^{-1} on X^T)
    TR_UPPER = 2         // P := U^{-1} P (backward substitution of the solve)
};
// Flag or-ed into TTrsm::mode: the task is not counted in the model flops (work the method itself
// does not do, such as forming the inverses of diagonal blocks for the solve).
constexpr int32_t kTrsmNoFlops = 0x100;

struct TGetrf {
    int64_t off;   // m x m column-major, ld = m
    int32_t m;
    int32_t leaf;  // for error reports
};

struct TTrsm {
    int64_t L_off;  // m x m leaf, ld = m
    int32_t m;
    int32_t mode;
    Panel P;        // m x p
};

// T (k x p) = F^T X with F: len x k and X: len x p.  kdyn[dst0] = kdyn[src0],
// kdyn[dst1] = kdyn[src1] when the slots are >= 0 (snapshot of dynamic sizes).
struct TProject {
    Panel F, X, T;
    int32_t dst0, src0, dst1, src1;
    int32_t no_flops;  // 1: not counted in the model flops
    int32_t pad_;
};

// out (rows x p) = beta*out + alpha * sum_t A_t X_t, with A_t: rows x inner_t,
// X_t: inner_t x p.  beta = 0 when overwrite.  kdyn[dst] = kdyn[src] if dst >= 0.
// Model flops: 2 rows inner p when credit == 0; credit * p when credit > 0 (a product that stands
// in for other operations of the method: those operations' count); none when credit < 0.
struct TAccum {
    Panel out;
    double alpha;
    int32_t overwrite;
    int32_t term0, nterms;
    int32_t dst, src;
    float credit;
};

struct Term {
    Panel A, X;
};

// Target low-rank block (m x n) with factors U (m x cap, ld m) and V (n x cap,
// ld n) and rank kdyn[kslot].  New value = T_eps(self + sum_i coef_i U_i V_i^T)
// where piece i covers target rows [roff, roff+rows(U_i)) and columns
// [coff, coff+rows(V_i)) (zero elsewhere); self is omitted if !include_self.
struct TRadd {
    int64_t U_off, V_off;
    int64_t scratch_off;   // (m + n) x Kcap workspace in the arena
    int32_t m, n;
    int32_t cap, kslot;
    int32_t include_self;
    int32_t piece0, npieces;
    int32_t Kcap;
    int32_t target;        // block id for error reports
    int32_t inst;          // instance of a batch (index into the per-instance tolerances), else 0
};

struct Piece {
    double coef;
    Panel U, V;
    int32_t roff, coff;
};

// dst U (mu x k) = src U rows, dst V (nv x k) = src V rows, kdyn[dst_kslot] = kdyn[src_kslot]
struct TSplit {
    Panel srcU, srcV;
    int64_t dstU, dstV;
    int32_t mu, nv;
    int32_t src_kslot, dst_kslot;
};

// Error word layout (device, int64[4]): code, index, value bits, count.
enum DevErr : int32_t {
    DE_OK = 0,
    DE_PIVOT = 1,
    DE_RANKCAP = 2,
    DE_NONFINITE = 3,
    DE_TIMEOUT = 4
};

}  // namespace hlu
