// Internal types shared by the planner (host) and the executor.  Not part of the ABI.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/ustat.h"

namespace ustat {

constexpr int kMaxM = 7;        // Bell(7) = 877 partitions
constexpr int kMaxTerms = 4;    // matrix terms read by one elementwise / reduce op
constexpr int kMaxScal = 6;     // scalar slots multiplied into one V_pi

// One factor matrix read with an orientation: value(i, j) = M[i][j] (trans = 0)
// or M[j][i] (trans = 1).
struct Term {
    int mat = -1;
    int trans = 0;
    bool operator==(const Term &o) const { return mat == o.mat && trans == o.trans; }
    bool operator<(const Term &o) const { return mat != o.mat ? mat < o.mat : trans < o.trans; }
};

enum OpKind : int {
    OP_KBUILD = 0,   // mat out = kernel map of factor f on X (RBF / LINEAR)
    OP_LOADMAT,      // mat out = caller matrix of factor f (converted to the working type)
    OP_UNARY,        // vec out = tanh(X w) of factor f
    OP_LOADVEC,      // vec out = caller vector of factor f
    OP_DIAG,         // vec out(i) = M(i, i) of t[0]
    OP_VMUL,         // vec out = u[0] * u[1] (elementwise)
    OP_HADAMARD,     // mat out(i, j) = prod_t t[t](i, j)
    OP_GEMV,         // vec out(j) = sum_i u(i) prod_t t[t](i, j)
    OP_VSUM,         // scal out += sum_i u(i)
    OP_GEMM,         // mat out(j, k) = sum_i A(i, j) u(i) B(i, k)
    OP_GEMM_RED,     // scal out += sum_jk [sum_i A(i,j) u(i) B(i,k)] W(j,k) a(j) b(k)
    OP_FREDUCE,      // scal out += sum_jk prod_t t[t](j, k) a(j) b(k)
    OP_GEMM3,        // scal out += sum_b ub(b) sum_cd [sum_a u(a) Ab(a,b) A(a,c) B(a,d)]
                     //             W(c,d) Wbc(b,c) Wbd(b,d) a(c) b(d)
    OP_SPLIT,        // operand out = bf16x3 fixed-point slices of the K-major operand
                     //   X(j, i) = t[0](i, j) u(i)
    OP_PREP,         // operand out = fp32 K-major copy X(j, i) = t[0](i, j) u(i) (tf32-rounded)
    OP_MHB,          // several FREDUCE / GEMV ops over the same matrices in one pass
    OP_VDOT,         // scal out += sum_i u(i) a(i)
    OP_COUNT
};

const char *op_name(int kind);

// A reduction fused into a GEMM: out += sum_jk C(j,k)^pow W(j,k) a(j) b(k).
struct Red {
    Term W;
    int a = -1, b = -1, pow = 1, out = -1;
};
constexpr int kMaxRed = 4;

struct Op {
    int kind = 0;
    int factor = -1;
    int out = -1;                 // slot written
    int store = 1;                // GEMM: write the product to `out`
    int nred = 0;                 // GEMM / KBUILD: fused reductions (KBUILD: red[r].pow
                                  // and red[r].out only; a vector out takes row sums)
    Red red[kMaxRed];
    int symmetric = 0;            // GEMM: product and reductions symmetric (upper tiles only)
    Term t[kMaxTerms];
    int nt = 0;
    int u = -1, a = -1, b = -1;   // vector slots (-1 = all ones)
    Term A, B, W;                 // GEMM operands / weight (W.mat = -1 = all ones)
    int opA = -1, opB = -1;       // operand slots for tensor-core GEMMs (SPLIT / PREP outputs)
    // GEMM3 only
    Term Ab, Wbc, Wbd;
    int ub = -1;
    double flops = 0.0;           // algorithmic flops per unit n-power (set by the planner)
    int npow = 0;                 // flops = coef * n^npow
    double coef = 0.0;
    int group = -1;               // OP_MHB: index into Plan::groups
    int upper_only = 0;           // KBUILD: its matrix is read only on and above the diagonal
};

enum SlotKind : int { S_MAT = 0, S_VEC, S_SCAL, S_SLICES, S_PREP };

struct Slot {
    int kind = S_MAT;
    int symmetric = 0;            // matrices only
};

struct PartRec {
    int rgs[kMaxM];
    int nblocks = 0;
    int mu = 0;
    int tw = -1;                  // exact treewidth of G/pi (simple quotient graph)
    int evaluated = 1;            // 0: skipped by sparsification or left to another shard (V = 0)
    int nfree = 0;                // blocks with no factor at all: factor n each
    int nscal = 0;
    int scal[kMaxScal];
    double naive_coef[5] = {0, 0, 0, 0, 0};   // own elimination cost: sum coef * n^p
    int order[kMaxM] = {-1, -1, -1, -1, -1, -1, -1};   // elimination order of the quotient's blocks
};

struct Plan {
    int m = 0;
    int precision = USTAT_FP64;
    int sparsify = 0;
    int planner = USTAT_PLAN_EXHAUSTIVE;
    int cse = 1;
    std::vector<int> factor_kind;   // per factor id
    std::vector<Slot> slots;
    std::vector<Op> ops;
    std::vector<std::vector<Op>> groups;   // members of OP_MHB operations
    std::vector<PartRec> parts;
    int n_gemm = 0, n_gemm3 = 0;
    // kernel variant per size class (tc_size_class): bits 0-1 = raster group index
    // into kGroupRows, bits 2-3 = GEMM tile shape (launch_gemm_bf16x3 / _bf16x4),
    // bit 4 = 64 x 64 tiles in the RBF kernel-matrix build; set by the batched
    // autotuner or ustat_plan_set_variant
    int tc_variant[4] = {0, 0, 0, 0};
};

constexpr int kGroupRows[4] = {8, 4, 16, 2};
inline int tc_size_class(int64_t n) { return n <= 1024 ? 0 : (n <= 2048 ? 1 : (n <= 3072 ? 2 : 3)); }

inline bool is_split_mode(int precision) {
    return precision == USTAT_BF16X3 || precision == USTAT_BF16X4 || precision == USTAT_BF16X5;
}
inline bool is_tc_mode(int precision) { return is_split_mode(precision) || precision == USTAT_TF32; }
inline int split_planes_of(int precision) {
    return precision == USTAT_BF16X5 ? 5 : (precision == USTAT_BF16X4 ? 4 : 3);
}
// matrices are stored in float64 in the FP64 mode and in the bf16x4 mode (whose
// purpose is data of wide dynamic range: float32 storage would round the few
// entries that dominate such sums), in float32 otherwise
inline bool wide_storage(int precision) {
    return precision == USTAT_FP64 || precision == USTAT_BF16X4 || precision == USTAT_BF16X5;
}

// Features of one candidate elimination sequence of one partition, for the
// learned order ranker (see order_features in planner.cpp).
constexpr int kRankFeatures = 20;
struct Candidate {
    std::vector<int> order;   // block ids of the quotient, elimination order
    float feat[kRankFeatures];
};

// Optional inputs / outputs of build_plan.
struct PlanRequest {
    // per partition (restricted-growth-string order): an elimination order to use
    // instead of the planner's search (empty: search)
    const std::vector<std::vector<int>> *forced = nullptr;
    // evaluate only the partition with m blocks (every vertex distinct): the plan
    // of the kernel graph's own contraction; the others are reported as 0
    bool finest_only = false;
    // if set: evaluate only the partitions whose entry is nonzero (a shard of the
    // partition sum); the others are reported as 0
    const std::vector<char> *keep = nullptr;
    // if set: every evaluated partition's distinct elimination sequences with
    // their features at sample size n (the plan is built as usual)
    std::vector<std::vector<Candidate>> *collect = nullptr;
    int collect_part = -1;   // >= 0: collect for this partition only
    bool collect_only = false;   // stop after collecting (no plan)
    // if set (with collect_part >= 0): the features of this one order of that
    // partition instead of the candidate list
    const std::vector<int> *feature_order = nullptr;
    int64_t n = 1024;
    // lower the partitions from the finest down (the sharing-aware search then
    // meets the partitions that need the most products first)
    bool reverse = false;
};

// Planner entry (planner.cpp).  Returns a USTAT_* code.
int build_plan(const ustat_graph *g, const ustat_options *o, Plan *plan, const PlanRequest *req = nullptr);

// Records a CUDA error for ustat_last_cuda_error and returns USTAT_ERR_CUDA (api.cu).
int record_cuda_error(int cuda_error);
// The USTAT_* status that an evaluation's device error word stands for (api.cu).
int status_of_word(int word);

// Exact treewidth of a simple graph on k <= 16 vertices given as adjacency bitmasks.
int exact_treewidth(int k, const std::vector<uint32_t> &adj);

}  // namespace ustat

struct ustat_plan {
    ustat::Plan p;
};
