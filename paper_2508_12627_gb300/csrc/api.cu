// C ABI (include/ustat.h): plans, workspace layout and the executor that walks
// a plan's lowered program and launches one kernel per operation on the
// caller's stream, ending with the Moebius combination (Algorithm 4).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "kernels.h"
#include "ustat_internal.h"

using namespace ustat;

namespace {

thread_local std::string g_last_cuda_error;

int cuda_fail(cudaError_t e) {
    g_last_cuda_error = cudaGetErrorString(e);
    return USTAT_ERR_CUDA;
}

// ---- optional per-operation event timing (ustat_profile_*)
constexpr int kProfXconvert = OP_COUNT, kProfCombine = OP_COUNT + 1, kProfKinds = OP_COUNT + 2;
struct ProfRec {
    int kind;
    cudaEvent_t a, b;
    int kernels;
};
struct Profiler {
    bool on = false;
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    std::vector<ProfRec> recs;
    cudaEvent_t get() {
        if (used == pool.size()) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
            pool.push_back(e);
        }
        return pool[used++];
    }
};
thread_local Profiler g_prof;

struct ProfScope {
    cudaStream_t st;
    ProfRec r{-1, nullptr, nullptr, 1};
    int kernels = 1;   // kernel launches of the operation (set by operations that make several)
    ProfScope(int kind, cudaStream_t s) : st(s) {
        if (!g_prof.on) return;
        r.kind = kind;
        r.a = g_prof.get();
        r.b = g_prof.get();
        if (r.a) cudaEventRecord(r.a, st);
    }
    ~ProfScope() {
        if (r.kind < 0 || !r.a || !r.b) return;
        cudaEventRecord(r.b, st);
        r.kernels = kernels;
        g_prof.recs.push_back(r);
    }
};

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct Layout {
    std::vector<size_t> off;     // per slot
    std::vector<int> scal_index; // per slot: index into the scalar array (or -1)
    size_t err_off = 0, scal_off = 0, zero_bytes = 0, xw_off = 0, total = 0;
    size_t kb_off = 0;   // scratch of the tensor-core RBF build (X digits, scales, norms)
    // float64-storage modes with s = 3 steps: float copies of one step's A source
    // (hi, lo) and of its weights W, Wbc, Wbd, for the float32 split and epilogue
    size_t sh_off = 0;
    int64_t ldp_slices = 0, ldp_prep = 0;
    // s = 3 steps on the tensor cores: digit planes of g3_nb A operands at a time
    size_t g3_off = 0, g3_stride = 0;
    int g3_nb = 0;
    int g3_regions = 1;
};

bool tc_gemm3(const Plan &P) {
    if (!is_split_mode(P.precision)) return false;
    for (auto &op : P.ops)
        if (op.kind == OP_GEMM3) return true;
    return false;
}

// an RBF kernel matrix built in float32 (the tensor-core Gram build's scratch)
bool has_rbf_f32_build(const Plan &P) {
    if (wide_storage(P.precision)) return false;
    for (auto &op : P.ops)
        if (op.kind == OP_KBUILD && op.factor >= 0 && P.factor_kind[op.factor] == USTAT_RBF) return true;
    return false;
}

bool needs_xw(const Plan &P) {
    for (auto &op : P.ops)
        if (op.kind == OP_KBUILD) return true;
    return false;
}

Layout make_layout(const Plan &P, int64_t n, int d) {
    Layout L;
    const size_t esz = wide_storage(P.precision) ? 8 : 4;
    L.ldp_slices = (int64_t)align_up((size_t)n, 64);
    L.ldp_prep = (int64_t)align_up((size_t)n, 32);
    L.off.assign(P.slots.size(), 0);
    L.scal_index.assign(P.slots.size(), -1);
    size_t cur = 0;
    L.err_off = cur;
    cur += 256;
    L.scal_off = cur;
    int ns = 0;
    for (size_t s = 0; s < P.slots.size(); ++s)
        if (P.slots[s].kind == S_SCAL) {
            L.scal_index[s] = ns;
            L.off[s] = cur + 8 * (size_t)ns;
            ++ns;
        }
    cur = align_up(cur + 8 * (size_t)ns, 256);
    for (size_t s = 0; s < P.slots.size(); ++s)
        if (P.slots[s].kind == S_VEC) {
            L.off[s] = cur;
            cur = align_up(cur + 8 * (size_t)n, 256);
        }
    L.zero_bytes = cur;   // error word, scalars and vectors are cleared per evaluation
    cur = align_up(cur, 1024);
    if (needs_xw(P)) {
        L.xw_off = cur;
        cur = align_up(cur + esz * (size_t)n * d, 1024);
    }
    if (has_rbf_f32_build(P)) {
        L.kb_off = cur;
        cur = align_up(cur + kbuild_rbf_tc_scratch_bytes(n, d), 1024);
    }
    for (size_t s = 0; s < P.slots.size(); ++s) {
        switch (P.slots[s].kind) {
            case S_MAT:
                L.off[s] = cur;
                cur = align_up(cur + esz * (size_t)n * n, 1024);
                break;
            case S_SLICES:
                // digit planes, row scales, and the diagonal left out of the digits
                L.off[s] = cur;
                cur = align_up(cur + split_planes_of(P.precision) * 2 * (size_t)n * L.ldp_slices +
                                   align_up(4 * (size_t)n, 256) + 8 * (size_t)n,
                               1024);
                break;
            case S_PREP:
                L.off[s] = cur;
                cur = align_up(cur + 4 * (size_t)n * L.ldp_prep, 1024);
                break;
            default:
                break;
        }
    }
    if (tc_gemm3(P)) {
        // about 256 MiB of A operands per batch, 1 to 64 of them
        L.g3_stride = align_up(split_planes_of(P.precision) * 2 * (size_t)n * L.ldp_slices + 4 * (size_t)n, 1024);
        L.g3_nb = (int)std::max<size_t>(1, std::min<size_t>(64, ((size_t)256 << 20) / L.g3_stride));
        L.g3_nb = (int)std::min<int64_t>(L.g3_nb, n);
        L.g3_off = cur;
        // two regions when there is more than one batch: the next batch's
        // operands are split while the tensor cores work on the current one
        L.g3_regions = L.g3_nb < n ? 2 : 1;
        cur = align_up(cur + L.g3_stride * L.g3_nb * L.g3_regions, 1024);
        if (wide_storage(P.precision) && n <= kPairSplitMaxN) {
            L.sh_off = cur;
            cur = align_up(cur + 5 * align_up(4 * (size_t)n * n, 1024), 1024);
        }
    }
    L.total = cur;
    return L;
}

// A second stream, of the highest priority, and events per host thread and
// device: the GEMMs of the s = 3 batches run on it while the operand split of
// the next batch runs on the caller's stream.  At equal priority the split's
// many short CTAs would take every SM as the previous GEMM drains and keep the
// persistent GEMM waiting; with the GEMM first, the split fills what the GEMM's
// CTAs leave of each SM (registers and shared memory for two split CTAs).
// Every piece of work on the second stream is joined back into the caller's
// stream by an event, so the pair also records correctly into a CUDA graph
// capture of the caller's stream.
struct SideStream {
    int dev = -1;
    cudaStream_t st = nullptr;
    cudaEvent_t split_done[2] = {nullptr, nullptr}, gemm_done[2] = {nullptr, nullptr};
    ~SideStream() {
        if (dev < 0) return;
        int cur = -1;
        if (cudaGetDevice(&cur) != cudaSuccess || cur != dev) return;   // leave them to the context
        for (int h = 0; h < 2; ++h) {
            cudaEventDestroy(split_done[h]);
            cudaEventDestroy(gemm_done[h]);
        }
        cudaStreamDestroy(st);
    }
};
thread_local SideStream g_side[16];

cudaError_t side_stream(SideStream **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 16) return cudaErrorInvalidDevice;
    SideStream &S = g_side[dev];
    if (S.dev < 0) {
        int least = 0, greatest = 0;
        e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&S.st, cudaStreamNonBlocking, greatest);
        for (int h = 0; h < 2 && e == cudaSuccess; ++h) {
            e = cudaEventCreateWithFlags(&S.split_done[h], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S.gemm_done[h], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) return e;
        S.dev = dev;
    }
    *out = &S;
    return cudaSuccess;
}

struct Ctx {
    const Plan &P;
    const Layout &L;
    char *ws;
    int64_t n;
    int d;
    bool fp64;
    cudaStream_t st;
    // row shard (ustat_eval_rows): this rank's share of the n^3 reduction products
    // and of the treewidth-3 indices; nranks = 1 is a whole evaluation
    int rank = 0, nranks = 1;
    void *ptr(int slot) const { return slot < 0 ? nullptr : (void *)(ws + L.off[slot]); }
    double *vec(int slot) const { return (double *)ptr(slot); }
    // slices: [3][n][ldp] bf16 followed by float scales [n]
    float *scales(int slot) const {
        return (float *)(ws + L.off[slot] + split_planes_of(P.precision) * 2 * (size_t)n * L.ldp_slices);
    }
    double *diagv(int slot) const {
        return (double *)(ws + L.off[slot] + split_planes_of(P.precision) * 2 * (size_t)n * L.ldp_slices +
                          align_up(4 * (size_t)n, 256));
    }
};

// Diagonal correction of the split-mode products (Section 3.1's factor matrices
// of positive-definite kernels, and their entrywise powers, have dominant
// diagonals; a row scale set by the diagonal leaves the off-diagonal entries few
// digits).  A split slot may leave dominant diagonal entries out when every
// reader is a non-batched product both of whose operands are split slots; such a
// product adds the left-out terms exactly in its epilogue.
struct DiagFix {
    std::vector<int> split_op;   // per slot: the OP_SPLIT op writing it, or -1
    std::vector<char> removed;   // per slot: split with its diagonal left out
};

DiagFix diag_fix_of(const Plan &P, int64_t n) {
    DiagFix D;
    D.split_op.assign(P.slots.size(), -1);
    D.removed.assign(P.slots.size(), 0);
    // plan variant bit 7 turns the correction off for this size class
    if (!is_split_mode(P.precision) || ((P.tc_variant[tc_size_class(n)] >> 7) & 1)) return D;
    for (size_t i = 0; i < P.ops.size(); ++i)
        if (P.ops[i].kind == OP_SPLIT && P.ops[i].out >= 0) D.split_op[P.ops[i].out] = (int)i;
    std::vector<char> ok(P.slots.size(), 1);
    for (const Op &op : P.ops) {
        if (op.kind == OP_GEMM) {
            const bool both = op.opA >= 0 && op.opB >= 0 && D.split_op[op.opA] >= 0 && D.split_op[op.opB] >= 0;
            if (!both) {
                if (op.opA >= 0) ok[op.opA] = 0;
                if (op.opB >= 0) ok[op.opB] = 0;
            }
        } else if (op.kind == OP_GEMM3) {
            if (op.opA >= 0) ok[op.opA] = 0;
            if (op.opB >= 0) ok[op.opB] = 0;
        }
    }
    for (size_t sl = 0; sl < P.slots.size(); ++sl) D.removed[sl] = D.split_op[sl] >= 0 && ok[sl];
    return D;
}

int check_graph_factors(const Plan &P, const ustat_factor *f, int nf, int d) {
    if (nf != (int)P.factor_kind.size() || !f) return USTAT_ERR_INVALID_ARG;
    for (int i = 0; i < nf; ++i) {
        if (f[i].kind != P.factor_kind[i]) return USTAT_ERR_INVALID_ARG;
        int k = f[i].kind;
        if ((k == USTAT_RBF || k == USTAT_LINEAR) && !(f[i].param > 0.0)) return USTAT_ERR_INVALID_ARG;
        if ((k == USTAT_TANH_DOT || k == USTAT_MATRIX || k == USTAT_VECTOR || k == USTAT_DIST || k == USTAT_LOWRANK ||
             k == USTAT_COMPLEMENT || k == USTAT_GRAM) &&
            !f[i].data)
            return USTAT_ERR_INVALID_ARG;
        // DIST, LOWRANK and GRAM: param is the data's column count (a positive integer)
        if ((k == USTAT_DIST || k == USTAT_LOWRANK || k == USTAT_GRAM) &&
            !(f[i].param >= 1.0 && f[i].param <= 4096.0 && f[i].param == (double)(int)f[i].param))
            return USTAT_ERR_INVALID_ARG;
    }
    (void)d;
    return USTAT_OK;
}

// The Moebius combination of a plan's scalars (one warp, float64, compensated).
cudaError_t plan_combine(const Plan &P, const Layout &L, const double *scal, const int *err, int64_t n,
                         double *U_out, double *V_out, cudaStream_t st) {
    static thread_local std::vector<CombineEntry> tab;
    tab.resize(P.parts.size());
    for (size_t p = 0; p < P.parts.size(); ++p) {
        const PartRec &pr = P.parts[p];
        CombineEntry &en = tab[p];
        en.mu = pr.mu;
        en.nfree = (unsigned char)pr.nfree;
        en.evaluated = (unsigned char)pr.evaluated;
        for (int q = 0; q < kCombineMaxScal; ++q)
            en.sid[q] = (q < pr.nscal) ? (unsigned short)L.scal_index[pr.scal[q]] : (unsigned short)0xffff;
    }
    return launch_combine(tab.data(), (int)tab.size(), P.m, scal, err, n, U_out, V_out, st);
}

// Row shard: the scalar slots written by sharded work (the reductions of products
// that store nothing, computed on a range of their tiles, and the treewidth-3
// steps, computed on a range of indices); every other scalar is computed whole on
// every rank.  A plan whose steps read a scalar cannot be sharded this way.
bool row_shard_slots(const Plan &P, std::vector<char> &sharded) {
    sharded.assign(P.slots.size(), 0);
    auto is_scal = [&](int s) { return s >= 0 && P.slots[s].kind == S_SCAL; };
    for (const Op &op : P.ops) {
        if (is_scal(op.u) || is_scal(op.a) || is_scal(op.b) || is_scal(op.ub)) return false;
        for (int t = 0; t < op.nt; ++t)
            if (is_scal(op.t[t].mat)) return false;
    }
    const bool tc = is_split_mode(P.precision) || P.precision == USTAT_TF32;
    for (const Op &op : P.ops) {
        if (op.kind == OP_GEMM && tc && !op.store)
            for (int r = 0; r < op.nred; ++r)
                if (is_scal(op.red[r].out)) sharded[op.red[r].out] = 1;
        if (op.kind == OP_GEMM3 && is_split_mode(P.precision) && is_scal(op.out)) sharded[op.out] = 1;
    }
    return true;
}

// The per-evaluation state every step reads: the error word, whether the RBF
// builds read the caller's X directly, the split width and the diagonal
// correction of the plan's split slots.
struct ProgState {
    int *err = nullptr;
    bool direct_x = false;
    int lead = 0;
    DiagFix D;
};

// Clears the evaluation's scalars and vectors and converts X where a step needs it.
int program_prologue(const Ctx &C, const void *X, int x_dtype, const ustat_factor *f, ProgState &S) {
    const Plan &P = C.P;
    const int64_t n = C.n;
    cudaError_t e = cudaMemsetAsync(C.ws, 0, C.L.zero_bytes, C.st);
    if (e != cudaSuccess) return cuda_fail(e);
    S.err = (int *)(C.ws + C.L.err_off);
    // float32 storage with RBF builds only: they read the caller's X directly
    S.direct_x = !C.fp64;
    for (const Op &op : P.ops)
        if (op.kind == OP_KBUILD && f[op.factor].kind != USTAT_RBF) S.direct_x = false;
    if (needs_xw(P) && !S.direct_x) {
        ProfScope ps(kProfXconvert, C.st);
        e = launch_xconvert(X, x_dtype, n, C.d, C.ws + C.L.xw_off, C.fp64, S.err, C.st);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    S.lead = split_lead_bits(n);
    S.D = diag_fix_of(P, n);
    return USTAT_OK;
}

// The tensor-core GEMM arguments of one product step on one evaluation's
// workspace (all but the tile shape), and the shape its size class selects.
void tc_gemm_args(const Ctx &C, const Op &op, const ProgState &S, TcGemmArgs &g, int &shape) {
    const Plan &P = C.P;
    const int64_t n = C.n;
    int *err = S.err;
    const int lead = S.lead;
    const DiagFix &D = S.D;
    auto trW = [&](const Term &t) { return (t.mat >= 0 && !P.slots[t.mat].symmetric) ? t.trans : 0; };
    const bool split = is_split_mode(P.precision);
    g = TcGemmArgs{};
    g.n = n;
    g.ldp = split ? C.L.ldp_slices : C.L.ldp_prep;
    g.opA = C.ptr(op.opA);
    g.opB = C.ptr(op.opB);
    g.scaleA = split ? C.scales(op.opA) : nullptr;
    g.scaleB = split ? C.scales(op.opB) : nullptr;
    g.lead_bits = lead;
    g.err = err;
    g.C = op.store ? C.ptr(op.out) : nullptr;
    g.wide = C.fp64;
    g.nred = op.nred;
    for (int r = 0; r < op.nred; ++r) {
        const Red &R = op.red[r];
        g.red[r] = TcRed{C.ptr(R.W.mat), trW(R.W), C.vec(R.a), C.vec(R.b), R.pow,
                         (double *)C.ptr(R.out)};
    }
    g.symmetric = op.symmetric;
    if (C.nranks > 1 && !op.store) {
        g.shard_rank = C.rank;
        g.shard_count = C.nranks;
    }
    if (split && op.opA >= 0 && op.opB >= 0 && (D.removed[op.opA] || D.removed[op.opB])) {
        // operands split without their diagonal: the epilogue adds the
        // left-out terms from the operands' sources
        const Op &sa = P.ops[D.split_op[op.opA]], &sb = P.ops[D.split_op[op.opB]];
        const bool symA = P.slots[sa.t[0].mat].symmetric, symB = P.slots[sb.t[0].mat].symmetric;
        const int trA = symA ? 1 : sa.t[0].trans, trB = symB ? 1 : sb.t[0].trans;
        g.dA = D.removed[op.opA] ? C.diagv(op.opA) : nullptr;
        g.dB = D.removed[op.opB] ? C.diagv(op.opB) : nullptr;
        g.MA = C.ptr(sa.t[0].mat);
        g.MB = C.ptr(sb.t[0].mat);
        // a symmetric source is read as M[k][j]: consecutive lanes (rows j)
        // then read consecutive addresses
        g.rowA = trA && !symA;
        g.rowB = !trB && !symB;
        g.uA = C.vec(sa.u);
        g.uB = C.vec(sb.u);
    }
    const int var = P.tc_variant[tc_size_class(n)];
    g.group_rows = kGroupRows[var & 3];
    shape = (var >> 2) & 3;
    if (shape == 1 && op.symmetric) shape = 0;   // 128 x 64 tiles cannot skip symmetric tiles
}

// One step of a plan on one evaluation's workspace.
int run_op(const Ctx &C, const Op &op, const ProgState &S, const void *X, int x_dtype, const ustat_factor *f) {
    const Plan &P = C.P;
    const int64_t n = C.n;
    int *err = S.err;
    const int lead = S.lead;
    const DiagFix &D = S.D;
    const bool direct_x = S.direct_x;
    cudaError_t e = cudaSuccess;
    ProfScope ps(op.kind, C.st);
    switch (op.kind) {
        case OP_KBUILD:
            if (!C.fp64 && f[op.factor].kind == USTAT_RBF) {
                int rpow[kMaxRed], rvec[kMaxRed];
                double *rout[kMaxRed];
                for (int r = 0; r < op.nred; ++r) {
                    rpow[r] = op.red[r].pow;
                    rvec[r] = P.slots[op.red[r].out].kind == S_VEC;
                    rout[r] = C.vec(op.red[r].out);   // scalar and vector slots are float64
                }
                const int var = P.tc_variant[tc_size_class(n)];
                if (!((var >> 5) & 1) && C.d <= 256) {
                    // default: squared distances from the Gram matrix on the tensor cores
                    e = launch_kbuild_rbf_tc(X, x_dtype, n, C.d, f[op.factor].param, P.sparsify,
                                             (float *)C.ptr(op.out), op.opA >= 0 ? C.ptr(op.opA) : nullptr,
                                             C.L.ldp_slices, lead, split_planes_of(P.precision),
                                             op.opA >= 0 ? C.scales(op.opA) : nullptr, op.nred, rpow, rvec, rout,
                                             op.upper_only, C.ws + C.L.kb_off, err, C.st);
                    ps.kernels = 2;
                    break;
                }
                // variant bit 5: direct differences on the CUDA cores
                const float *xf = direct_x ? (x_dtype == 1 ? (const float *)X : nullptr)
                                           : (const float *)(C.ws + C.L.xw_off);
                const double *xd = direct_x && x_dtype == 0 ? (const double *)X : nullptr;
                e = launch_kbuild_rbf(xf, xd, n, C.d, f[op.factor].param, P.sparsify,
                                      (float *)C.ptr(op.out), op.opA >= 0 ? C.ptr(op.opA) : nullptr,
                                      C.L.ldp_slices, lead, split_planes_of(P.precision),
                                      op.opA >= 0 ? C.scales(op.opA) : nullptr, op.nred, rpow, rvec, rout,
                                      op.upper_only, (var >> 4) & 1, err, C.st);
            } else {
                if (op.nred) return USTAT_ERR_UNSUPPORTED;   // the planner fuses only into the RBF build
                if (C.fp64 && f[op.factor].kind == USTAT_LINEAR && x_dtype == 1)
                    e = launch_kbuild_linear_wide((const float *)X, n, C.d, f[op.factor].param, P.sparsify,
                                                  (double *)C.ptr(op.out), C.st);
                else
                    e = launch_kbuild(f[op.factor].kind, f[op.factor].param, C.ws + C.L.xw_off, C.fp64, n, C.d,
                                      P.sparsify, C.ptr(op.out), C.st);
            }
            break;
        case OP_LOADMAT:
            if (f[op.factor].kind == USTAT_DIST || f[op.factor].kind == USTAT_LOWRANK ||
                f[op.factor].kind == USTAT_GRAM)
                e = launch_pairs(f[op.factor].kind, (const double *)f[op.factor].data, (int)f[op.factor].param, n,
                                 C.fp64, P.sparsify, C.ptr(op.out), err, C.st);
            else
                e = launch_loadmat((const double *)f[op.factor].data, n, C.fp64, P.sparsify,
                                   f[op.factor].kind == USTAT_COMPLEMENT, C.ptr(op.out), err, C.st);
            break;
        case OP_UNARY:
            e = launch_unary_tanh(X, x_dtype, n, C.d, (const double *)f[op.factor].data, C.vec(op.out), err, C.st);
            break;
        case OP_LOADVEC:
            e = launch_copyvec((const double *)f[op.factor].data, n, C.vec(op.out), err, C.st);
            break;
        case OP_DIAG:
            if (op.factor >= 0 && f[op.factor].kind != USTAT_TANH_DOT && f[op.factor].kind != USTAT_VECTOR)
                e = launch_factor_diag(f[op.factor].kind, f[op.factor].param, X, x_dtype, C.d,
                                       (const double *)f[op.factor].data, n, P.sparsify, C.vec(op.out), C.st);
            else
                e = launch_diag(C.ptr(op.t[0].mat), C.fp64, n, C.vec(op.out), C.st);
            break;
        case OP_VMUL:
            e = launch_vmul(C.vec(op.u), C.vec(op.a), n, C.vec(op.out), C.st);
            break;
        case OP_VSUM:
            e = launch_vsum(C.vec(op.u), n, C.vec(op.out), C.st);
            break;
        case OP_VDOT:
            e = launch_vdot(C.vec(op.u), C.vec(op.a), n, C.vec(op.out), C.st);
            break;
        case OP_HADAMARD:
        case OP_GEMV:
        case OP_FREDUCE: {
            TileTerms tt{};
            tt.nt = op.nt;
            for (int t = 0; t < op.nt; ++t) {
                tt.M[t] = C.ptr(op.t[t].mat);
                tt.trans[t] = P.slots[op.t[t].mat].symmetric ? 0 : op.t[t].trans;
            }
            if (op.kind == OP_HADAMARD)
                e = launch_tile_op(TILE_HADAMARD, tt, C.fp64, n, nullptr, nullptr, C.ptr(op.out), C.st);
            else if (op.kind == OP_GEMV)
                e = launch_tile_op(TILE_GEMV, tt, C.fp64, n, C.vec(op.u), nullptr, C.ptr(op.out), C.st);
            else
                e = launch_tile_op(TILE_FREDUCE, tt, C.fp64, n, C.vec(op.a), C.vec(op.b), C.ptr(op.out), C.st);
            break;
        }
        case OP_MHB: {
            MhbArgs g{};
            g.n = n;
            std::vector<int> mats;
            auto mat_index = [&](int slot) {
                for (size_t q = 0; q < mats.size(); ++q)
                    if (mats[q] == slot) return (int)q;
                mats.push_back(slot);
                return (int)mats.size() - 1;
            };
            const auto &grp = P.groups[op.group];
            g.nops = (int)grp.size();
            for (size_t q = 0; q < grp.size(); ++q) {
                const Op &m = grp[q];
                MhbOp &h = g.op[q];
                h.kind = m.kind == OP_GEMV ? TILE_GEMV : TILE_FREDUCE;
                h.nt = m.nt;
                for (int t = 0; t < m.nt; ++t) h.mat[t] = mat_index(m.t[t].mat);
                h.a = m.kind == OP_GEMV ? C.vec(m.u) : C.vec(m.a);
                h.b = m.kind == OP_GEMV ? nullptr : C.vec(m.b);
                h.out = (double *)C.ptr(m.out);
            }
            if (mats.size() > (size_t)kMhbMats) return USTAT_ERR_UNSUPPORTED;
            g.nmat = (int)mats.size();
            for (size_t q = 0; q < mats.size(); ++q) g.M[q] = C.ptr(mats[q]);
            e = launch_mhb(g, C.fp64, C.st);
            break;
        }
        case OP_SPLIT:
        case OP_PREP: {
            const Term t = op.t[0];
            const int tr = P.slots[t.mat].symmetric ? 1 : t.trans;
            if (op.kind == OP_SPLIT) {
                double *dg = D.removed[op.out] ? C.diagv(op.out) : nullptr;
                e = launch_split(C.ptr(t.mat), C.fp64, tr, C.vec(op.u), n, C.L.ldp_slices, lead,
                                 split_planes_of(P.precision), C.ptr(op.out), C.scales(op.out), dg, C.st);
                if (dg) ps.kernels = 2;
            }
            else
                e = launch_prep((const float *)C.ptr(t.mat), tr, C.vec(op.u), n, C.L.ldp_prep,
                                (float *)C.ptr(op.out), C.st);
            break;
        }
        case OP_GEMM: {
            auto trW = [&](const Term &t) { return (t.mat >= 0 && !P.slots[t.mat].symmetric) ? t.trans : 0; };
            if (is_tc_mode(P.precision)) {
                TcGemmArgs g;
                int shape = 0;
                tc_gemm_args(C, op, S, g, shape);
                if (P.precision == USTAT_BF16X3) e = launch_gemm_bf16x3(g, shape, C.st);
                else if (P.precision == USTAT_BF16X4) e = launch_gemm_bf16x4(g, shape, C.st);
                else if (P.precision == USTAT_BF16X5) e = launch_gemm_bf16x5(g, C.st);
                else e = launch_gemm_tf32(g, C.st);
            } else {
                SimtGemmArgs g{};
                g.n = n;
                g.A = C.ptr(op.A.mat);
                g.transA = trW(op.A);
                g.B = C.ptr(op.B.mat);
                g.transB = trW(op.B);
                g.u = C.vec(op.u);
                g.C = op.store ? C.ptr(op.out) : nullptr;
                g.nred = op.nred;
                for (int r = 0; r < op.nred; ++r) {
                    const Red &R = op.red[r];
                    g.red[r] = SimtRed{C.ptr(R.W.mat), trW(R.W), C.vec(R.a), C.vec(R.b), R.pow,
                                       (double *)C.ptr(R.out)};
                }
                g.symmetric = op.symmetric;
                e = launch_gemm_simt(g, C.fp64, C.st);
            }
            break;
        }
        case OP_GEMM3: {
            auto tr = [&](const Term &t) { return (t.mat >= 0 && !P.slots[t.mat].symmetric) ? t.trans : 0; };
            if (is_split_mode(P.precision)) {
                // tensor cores: g3_nb products at a time, their A operands split
                // per bb into the batch region (planes of all bb back to back)
                // (two regions: batch k is split into region k % 2 once the GEMM
                // of batch k - 2 has read it; its GEMM runs on the second stream
                // after that split, beside the split of batch k + 1)
                const int planes = split_planes_of(P.precision);
                const size_t plane_bytes = 2 * (size_t)n * C.L.ldp_slices;
                const int var = P.tc_variant[tc_size_class(n)];
                const bool two = C.L.g3_regions == 2;
                SideStream *S = nullptr;
                if (two) {
                    e = side_stream(&S);
                    if (e != cudaSuccess) break;
                }
                const cudaStream_t gs = two ? S->st : C.st;
                // float64 storage: the A source as a float pair and the weights as
                // float, so that neither the split nor the GEMM epilogue of this
                // step does float64 arithmetic per entry
                auto row_form = [&](const Term &t) { return P.slots[t.mat].symmetric ? 1 : t.trans; };
                const bool pair = C.fp64 && C.L.sh_off && row_form(op.A) == 1;
                float *shA = nullptr, *shAl = nullptr, *shW = nullptr, *shWbc = nullptr, *shWbd = nullptr;
                if (pair) {
                    const size_t sz = align_up(4 * (size_t)n * n, 1024);
                    char *sh = C.ws + C.L.sh_off;
                    shA = (float *)sh;
                    shAl = (float *)(sh + sz);
                    shW = (float *)(sh + 2 * sz);
                    shWbc = (float *)(sh + 3 * sz);
                    shWbd = (float *)(sh + 4 * sz);
                    e = launch_f64_pair((const double *)C.ptr(op.A.mat), n * n, shA, shAl, C.st);
                    if (e == cudaSuccess && op.W.mat >= 0)
                        e = launch_f64_pair((const double *)C.ptr(op.W.mat), n * n, shW, nullptr, C.st);
                    if (e == cudaSuccess && op.Wbc.mat >= 0)
                        e = launch_f64_pair((const double *)C.ptr(op.Wbc.mat), n * n, shWbc, nullptr, C.st);
                    if (e == cudaSuccess && op.Wbd.mat >= 0)
                        e = launch_f64_pair((const double *)C.ptr(op.Wbd.mat), n * n, shWbd, nullptr, C.st);
                    if (e != cudaSuccess) break;
                }
                int k = 0, last = 0;
                // a row shard takes the indices bb_lo .. bb_hi - 1
                const int64_t bb_lo = n * C.rank / C.nranks, bb_hi = n * (C.rank + 1) / C.nranks;
                for (int64_t bb0 = bb_lo; bb0 < bb_hi && e == cudaSuccess; bb0 += C.L.g3_nb, ++k) {
                    const int nb = (int)std::min<int64_t>(C.L.g3_nb, bb_hi - bb0);
                    const int h = two ? (k & 1) : 0;
                    char *sl = C.ws + C.L.g3_off + (size_t)h * C.L.g3_stride * C.L.g3_nb;
                    float *sc = (float *)(sl + planes * plane_bytes * C.L.g3_nb);
                    if (two && k >= 2) e = cudaStreamWaitEvent(C.st, S->gemm_done[h], 0);
                    if (e != cudaSuccess) break;
                    // symmetric sources are read along rows (A(i, j) = M[j][i])
                    if (pair)
                        e = launch_split_g3_pair(shA, shAl, C.vec(op.u), (const double *)C.ptr(op.Ab.mat),
                                                 row_form(op.Ab), bb0, nb, n, C.L.ldp_slices, lead, planes, sl,
                                                 sc, C.st);
                    else
                        e = launch_split_g3(C.ptr(op.A.mat), C.fp64, row_form(op.A), C.vec(op.u),
                                            C.ptr(op.Ab.mat), row_form(op.Ab), bb0, nb, n, C.L.ldp_slices, lead,
                                            planes, sl, sc, C.st);
                    if (e == cudaSuccess && two) e = cudaEventRecord(S->split_done[h], C.st);
                    if (e == cudaSuccess && two) e = cudaStreamWaitEvent(gs, S->split_done[h], 0);
                    if (e != cudaSuccess) break;
                    TcGemmArgs g{};
                    g.n = n;
                    g.ldp = C.L.ldp_slices;
                    g.opA = sl;
                    g.scaleA = sc;
                    g.opB = C.ptr(op.opB);
                    g.scaleB = C.scales(op.opB);
                    g.lead_bits = lead;
                    g.err = err;
                    g.nred = 1;
                    g.red[0] = TcRed{op.W.mat >= 0 && pair ? (const void *)shW : C.ptr(op.W.mat), tr(op.W),
                                     C.vec(op.a), C.vec(op.b), 1, (double *)C.ptr(op.out)};
                    // with the float copies the step runs in the float32-storage form of
                    // the kernel (two accumulator sets, overlapped epilogue) unless
                    // variant bit 6 keeps the four-accumulator layout
                    const bool four_acc = ((var >> 6) & 1) || P.precision == USTAT_BF16X5;
                    g.wide = C.fp64 && !(pair && !four_acc);
                    g.wide_f32 = pair && four_acc ? 1 : 0;
                    g.batch = nb;
                    g.bb0 = (int)bb0;
                    g.Wbc = op.Wbc.mat >= 0 && pair ? (const void *)shWbc : C.ptr(op.Wbc.mat);
                    g.transWbc = tr(op.Wbc);
                    g.Wbd = op.Wbd.mat >= 0 && pair ? (const void *)shWbd : C.ptr(op.Wbd.mat);
                    g.transWbd = tr(op.Wbd);
                    g.ub = C.vec(op.ub);
                    g.group_rows = kGroupRows[var & 3];
                    if (P.precision == USTAT_BF16X3) e = launch_gemm_bf16x3(g, (var >> 2) & 3, gs);
                    else if (P.precision == USTAT_BF16X5) e = launch_gemm_bf16x5(g, gs);
                    else e = launch_gemm_bf16x4(g, (var >> 2) & 3, gs);
                    if (e == cudaSuccess && two) e = cudaEventRecord(S->gemm_done[h], gs);
                    last = h;
                }
                // a split and a GEMM per batch, and the float copies of the step
                ps.kernels = 2 * k + (pair ? 1 + (op.W.mat >= 0) + (op.Wbc.mat >= 0) + (op.Wbd.mat >= 0) : 0);
                // join: the caller's stream waits for the last GEMM (the second
                // stream runs its GEMMs in order)
                if (e == cudaSuccess && two && k > 0) e = cudaStreamWaitEvent(C.st, S->gemm_done[last], 0);
                break;
            }
            SimtGemmArgs g{};
            g.n = n;
            g.gemm3 = 1;
            g.A = C.ptr(op.A.mat);
            g.transA = tr(op.A);
            g.B = C.ptr(op.B.mat);
            g.transB = tr(op.B);
            g.u = C.vec(op.u);
            g.Ab = C.ptr(op.Ab.mat);
            g.transAb = tr(op.Ab);
            g.nred = 1;
            g.red[0] = SimtRed{C.ptr(op.W.mat), tr(op.W), C.vec(op.a), C.vec(op.b), 1, (double *)C.ptr(op.out)};
            g.Wbc = C.ptr(op.Wbc.mat);
            g.transWbc = tr(op.Wbc);
            g.Wbd = C.ptr(op.Wbd.mat);
            g.transWbd = tr(op.Wbd);
            g.ub = C.vec(op.ub);
            e = launch_gemm_simt(g, C.fp64, C.st);
            break;
        }
        default:
            return USTAT_ERR_UNSUPPORTED;
    }
    if (e != cudaSuccess) return cuda_fail(e);
    return USTAT_OK;
}

int run_program(const Ctx &C, const void *X, int x_dtype, const ustat_factor *f, double *U_out, double *V_out,
                double *scal_out = nullptr) {
    const Plan &P = C.P;
    const int64_t n = C.n;
    ProgState S;
    int rc = program_prologue(C, X, x_dtype, f, S);
    if (rc != USTAT_OK) return rc;
    for (const Op &op : P.ops) {
        rc = run_op(C, op, S, X, x_dtype, f);
        if (rc != USTAT_OK) return rc;
    }
    int *err = S.err;
    cudaError_t e = cudaSuccess;
    if (scal_out) {
        // row shard: this rank's scalars; the ones every rank computes whole count
        // on rank 0 only, so that the ranks' arrays sum to the plan's scalars
        int ns = 0;
        for (size_t sl = 0; sl < P.slots.size(); ++sl) ns += P.slots[sl].kind == S_SCAL;
        e = cudaMemcpyAsync(scal_out, C.ws + C.L.scal_off, 8 * (size_t)ns, cudaMemcpyDeviceToDevice, C.st);
        if (e != cudaSuccess) return cuda_fail(e);
        if (C.rank != 0) {
            std::vector<char> sharded;
            row_shard_slots(P, sharded);
            for (size_t sl = 0; sl < P.slots.size() && e == cudaSuccess; ++sl)
                if (P.slots[sl].kind == S_SCAL && !sharded[sl])
                    e = cudaMemsetAsync(scal_out + C.L.scal_index[sl], 0, 8, C.st);
            if (e != cudaSuccess) return cuda_fail(e);
        }
        return USTAT_OK;
    }
    {
        ProfScope ps(kProfCombine, C.st);
        e = plan_combine(P, C.L, (const double *)(C.ws + C.L.scal_off), err, n, U_out, V_out, C.st);
    }
    if (e != cudaSuccess) return cuda_fail(e);
    return USTAT_OK;
}

// ---------------------------------------------------------------- memory-lean evaluation
// The tensorization step stores every pairwise factor as an n x n matrix, and the
// s = 2 products read the stored matrices (the space bound of Section 3.3's
// remark on space complexity and of the appendix on it: O(n^2) for the factors).
// The lean form stores none: for plans whose n^2 objects are RBF factor matrices
// (built on the tensor cores from X) read only by products that keep nothing but
// their fused reductions, it walks the products panel by panel.  For a row panel
// J and a column panel L of one product it builds the digit planes of the
// factor's rows J and rows L (and, when a reduction weighs by the factor, its
// float32 rows J) into two panel buffers, then runs the product's window (J, L):
// the same digits, the same accumulation per entry, the reductions summed in
// another order.  Memory O(panel x n); the factor rows of L are rebuilt once per
// panel J, an O(n^3 d / panel) build beside the O(n^3) products.
struct LeanPlan {
    bool ok = false;
    std::vector<int> kb_of;   // per slot: the RBF build op writing it (its matrix or digit planes), or -1
    bool need_k = false;      // a product's reduction weighs by the factor matrix
};

LeanPlan lean_plan(const Plan &P) {
    LeanPlan LP;
    if (P.precision != USTAT_BF16X3) return LP;
    LP.kb_of.assign(P.slots.size(), -1);
    for (size_t i = 0; i < P.ops.size(); ++i) {
        const Op &op = P.ops[i];
        switch (op.kind) {
            case OP_KBUILD:
                if (P.factor_kind[op.factor] != USTAT_RBF) return LP;
                if (op.out >= 0) LP.kb_of[op.out] = (int)i;
                if (op.opA >= 0) LP.kb_of[op.opA] = (int)i;
                break;
            case OP_GEMM: {
                if (op.store || op.opA < 0 || op.opB < 0 || LP.kb_of[op.opA] < 0 || LP.kb_of[op.opB] < 0)
                    return LP;
                if (op.symmetric && LP.kb_of[op.opA] != LP.kb_of[op.opB]) return LP;
                for (int r = 0; r < op.nred; ++r) {
                    const int w = op.red[r].W.mat;
                    if (w < 0) continue;
                    // the weight must be the A operand's factor (its rows J are built)
                    if (LP.kb_of[w] != LP.kb_of[op.opA] || !P.slots[w].symmetric) return LP;
                    LP.need_k = true;
                }
                break;
            }
            case OP_DIAG:
                if (op.factor < 0) return LP;
                break;
            case OP_UNARY:
            case OP_LOADVEC:
            case OP_VMUL:
            case OP_VSUM:
            case OP_VDOT:
                break;
            default:
                return LP;
        }
    }
    LP.ok = true;
    return LP;
}

struct LeanLayout {
    Layout L;   // error word, scalars and vectors as in the stored form; kb_off the build's X scratch
    size_t a_off = 0, a_sc = 0, b_off = 0, b_sc = 0, k_off = 0;
};

LeanLayout make_lean_layout(const Plan &P, int64_t n, int d, int64_t panel, bool need_k) {
    LeanLayout LL;
    LL.L = make_layout(P, n, d);   // only its scalar and vector part is used
    Layout &L = LL.L;
    size_t cur = align_up(L.zero_bytes, 1024);
    L.kb_off = cur;
    cur = align_up(cur + kbuild_rbf_tc_scratch_bytes(n, d), 1024);
    const size_t planes = (size_t)split_planes_of(P.precision) * 2 * (size_t)panel * L.ldp_slices;
    LL.a_off = cur;
    cur = align_up(cur + planes, 1024);
    LL.a_sc = cur;
    cur = align_up(cur + 4 * (size_t)panel, 1024);
    LL.b_off = cur;
    cur = align_up(cur + planes, 1024);
    LL.b_sc = cur;
    cur = align_up(cur + 4 * (size_t)panel, 1024);
    if (need_k) {
        LL.k_off = cur;
        cur = align_up(cur + 4 * (size_t)panel * n, 1024);
    }
    L.total = cur;
    return LL;
}

int run_lean(const Plan &P, const LeanPlan &LP, const LeanLayout &LL, char *ws, int64_t n, int d, int64_t panel,
             const void *X, int x_dtype, const ustat_factor *f, cudaStream_t st, double *U_out, double *V_out) {
    const Layout &L = LL.L;
    Ctx C{P, L, ws, n, d, false, st};
    cudaError_t e = cudaMemsetAsync(ws, 0, L.zero_bytes, st);
    if (e != cudaSuccess) return cuda_fail(e);
    int *err = (int *)(ws + L.err_off);
    void *scratch = ws + L.kb_off;
    const int lead = split_lead_bits(n);
    const int planes = split_planes_of(P.precision);
    const int64_t ldp = L.ldp_slices;
    void *Apl = ws + LL.a_off, *Bpl = ws + LL.b_off;
    float *Asc = (float *)(ws + LL.a_sc), *Bsc = (float *)(ws + LL.b_sc);
    float *Kp = LL.k_off ? (float *)(ws + LL.k_off) : nullptr;
    bool prepped = false;
    auto prep = [&]() -> cudaError_t {
        if (prepped) return cudaSuccess;
        prepped = true;
        return launch_gram_rbf_prep(X, x_dtype, n, d, scratch, err, st);
    };
    // rows r0 .. r0 + rows - 1 of factor `fi` into a panel: digit planes and scales,
    // the float32 rows too when K is given
    auto panel_build = [&](int fi, int64_t r0, int64_t rows, float *K, void *pl, float *sc) {
        return launch_gram_rbf_window(n, d, f[fi].param, P.sparsify, K ? K - r0 * n : nullptr, pl, ldp, lead, planes,
                                      sc - r0, 0, nullptr, nullptr, nullptr, r0, rows, 0, n, r0, rows * ldp, scratch,
                                      err, st);
    };
    const int var = P.tc_variant[tc_size_class(n)];
    for (const Op &op : P.ops) {
        ProfScope ps(op.kind, st);
        switch (op.kind) {
            case OP_KBUILD: {
                e = prep();
                if (e != cudaSuccess || op.nred == 0) break;
                // the build's fused reductions, panel by panel, nothing stored
                int rpow[kMaxRed], rvec[kMaxRed];
                double *rout[kMaxRed];
                for (int r = 0; r < op.nred; ++r) {
                    rpow[r] = op.red[r].pow;
                    rvec[r] = P.slots[op.red[r].out].kind == S_VEC;
                    rout[r] = C.vec(op.red[r].out);
                }
                for (int64_t r0 = 0; r0 < n && e == cudaSuccess; r0 += panel)
                    e = launch_gram_rbf_window(n, d, f[op.factor].param, P.sparsify, nullptr, nullptr, ldp, lead,
                                               planes, nullptr, op.nred, rpow, rvec, rout, r0,
                                               std::min(panel, n - r0), 0, n, 0, 0, scratch, err, st);
                break;
            }
            case OP_GEMM: {
                e = prep();
                const int fa = P.ops[LP.kb_of[op.opA]].factor, fb = P.ops[LP.kb_of[op.opB]].factor;
                bool weighted = false;
                for (int r = 0; r < op.nred; ++r) weighted |= op.red[r].W.mat >= 0;
                int shape = (var >> 2) & 3;
                if (shape == 1 && op.symmetric) shape = 0;
                for (int64_t r0 = 0; r0 < n && e == cudaSuccess; r0 += panel) {
                    const int64_t rj = std::min(panel, n - r0);
                    e = panel_build(fa, r0, rj, weighted ? Kp : nullptr, Apl, Asc);
                    for (int64_t c0 = op.symmetric ? r0 : 0; c0 < n && e == cudaSuccess; c0 += panel) {
                        const int64_t rl = std::min(panel, n - c0);
                        const bool same = c0 == r0 && fa == fb;
                        if (!same) e = panel_build(fb, c0, rl, nullptr, Bpl, Bsc);
                        if (e != cudaSuccess) break;
                        TcGemmArgs g{};
                        g.n = n;
                        g.ldp = ldp;
                        g.opA = Apl;
                        g.scaleA = Asc - r0;
                        g.opB = same ? Apl : Bpl;
                        g.scaleB = (same ? Asc : Bsc) - c0;
                        g.lead_bits = lead;
                        g.err = err;
                        g.nred = op.nred;
                        for (int r = 0; r < op.nred; ++r) {
                            const Red &R = op.red[r];
                            g.red[r] = TcRed{R.W.mat >= 0 ? (const void *)(Kp - r0 * n) : nullptr, 0, C.vec(R.a),
                                             C.vec(R.b), R.pow, (double *)C.ptr(R.out)};
                        }
                        g.symmetric = op.symmetric && c0 == r0;
                        g.wscale = (op.symmetric && c0 != r0) ? 2.0 : 1.0;   // the mirror window
                        g.row0 = r0;
                        g.rows = rj;
                        g.col0 = c0;
                        g.cols = rl;
                        g.group_rows = kGroupRows[var & 3];
                        e = launch_gemm_bf16x3(g, shape, st);
                    }
                }
                break;
            }
            case OP_UNARY:
                e = launch_unary_tanh(X, x_dtype, n, d, (const double *)f[op.factor].data, C.vec(op.out), err, st);
                break;
            case OP_LOADVEC:
                e = launch_copyvec((const double *)f[op.factor].data, n, C.vec(op.out), err, st);
                break;
            case OP_DIAG:
                e = launch_factor_diag(f[op.factor].kind, f[op.factor].param, X, x_dtype, d,
                                       (const double *)f[op.factor].data, n, P.sparsify, C.vec(op.out), st);
                break;
            case OP_VMUL:
                e = launch_vmul(C.vec(op.u), C.vec(op.a), n, C.vec(op.out), st);
                break;
            case OP_VSUM:
                e = launch_vsum(C.vec(op.u), n, C.vec(op.out), st);
                break;
            case OP_VDOT:
                e = launch_vdot(C.vec(op.u), C.vec(op.a), n, C.vec(op.out), st);
                break;
            default:
                return USTAT_ERR_UNSUPPORTED;
        }
        if (e != cudaSuccess) return cuda_fail(e);
    }
    {
        ProfScope ps(kProfCombine, st);
        e = plan_combine(P, L, (const double *)(ws + L.scal_off), err, n, U_out, V_out, st);
    }
    if (e != cudaSuccess) return cuda_fail(e);
    return USTAT_OK;
}

}  // namespace

int ustat::record_cuda_error(int e) { return cuda_fail((cudaError_t)e); }

// The status an evaluation's error word stands for: a bounded wait that gave up
// first, then a non-finite input.
int ustat::status_of_word(int word) {
    if (word & kErrWordTimeout) return USTAT_ERR_DEVICE_TIMEOUT;
    if (word & kErrWordNonfinite) return USTAT_ERR_NONFINITE;
    return USTAT_OK;
}

namespace {

// Modelled flops of a lowered program at sample size n.
double plan_model_flops(const Plan &P, double n) {
    double f = 0.0;
    for (auto &op : P.ops) f += op.coef * std::pow(n, op.npow);
    return f;
}

std::vector<std::vector<int>> plan_orders_of(const Plan &P) {
    std::vector<std::vector<int>> orders(P.parts.size());
    for (size_t pi = 0; pi < P.parts.size(); ++pi)
        for (int i = 0; i < kMaxM; ++i)
            if (P.parts[pi].order[i] >= 0) orders[pi].push_back(P.parts[pi].order[i]);
    return orders;
}

// The exhaustive planner with sharing chooses each partition's order greedily, in
// partition order, by the work it adds to the program built so far; that can
// commit early partitions to products later ones do not share (path + chord:
// six distinct n^3 products where two suffice).  The same search from the finest
// partition down is the second candidate (the finest partitions need the most
// products, and coarser ones then reuse them).  A bounded local search follows:
// for each partition in turn, each of its distinct elimination sequences is tried
// with every other partition's order kept, and a change is kept when the whole
// plan's modelled flops (at n = 8192, where the n^3 and n^4 terms decide) fall;
// two sweeps at most, and only for plans of at least two n^3 steps and at most
// 1000 candidate sequences in all (about 2 ms per trial plan).  Float32-storage
// modes only (see below).
int build_plan_best(const ustat_graph *g, const ustat_options *o, Plan *out) {
    int rc = build_plan(g, o, out);
    if (rc != USTAT_OK || o->planner != USTAT_PLAN_EXHAUSTIVE || !o->cse) return rc;
    // the float64-storage modes keep the greedy plan: on path + chord the cheaper
    // plan reduces against the stored product K K where the greedy one fuses those
    // reductions into products with K o K, and its bf16x4 result measured 6.7e-8 of
    // V_abs against 1.8e-9 (the storage's accuracy is what those modes are for)
    if (wide_storage(o->precision)) return rc;
    {
        // the same search from the finest partition down
        PlanRequest rreq;
        rreq.reverse = true;
        Plan rev;
        if (build_plan(g, o, &rev, &rreq) == USTAT_OK &&
            plan_model_flops(rev, 8192.0) < plan_model_flops(*out, 8192.0) * (1.0 - 1e-9))
            *out = std::move(rev);
    }
    int heavy = 0;
    for (const Op &op : out->ops) heavy += op.kind == OP_GEMM || op.kind == OP_GEMM3;
    if (heavy < 2) return rc;
    std::vector<std::vector<Candidate>> cands;
    PlanRequest creq;
    creq.collect = &cands;
    creq.n = 8192;
    Plan tmp;
    if (build_plan(g, o, &tmp, &creq) != USTAT_OK) return rc;
    size_t total = 0;
    for (auto &c : cands) total += c.size();
    if (total > 1000 || cands.size() != out->parts.size()) return rc;
    std::vector<std::vector<int>> orders = plan_orders_of(*out);
    double best = plan_model_flops(*out, 8192.0);
    for (int sweep = 0; sweep < 2; ++sweep) {
        bool improved = false;
        for (size_t pi = 0; pi < cands.size(); ++pi) {
            if (cands[pi].size() < 2) continue;
            for (const Candidate &cd : cands[pi]) {
                if (cd.order == orders[pi]) continue;
                std::vector<std::vector<int>> trial = orders;
                trial[pi] = cd.order;
                PlanRequest req;
                req.forced = &trial;
                Plan alt;
                if (build_plan(g, o, &alt, &req) != USTAT_OK) continue;
                const double f = plan_model_flops(alt, 8192.0);
                if (f < best * (1.0 - 1e-9)) {
                    best = f;
                    orders = std::move(trial);
                    *out = std::move(alt);
                    improved = true;
                }
            }
        }
        if (!improved) break;
    }
    return USTAT_OK;
}

}  // namespace

extern "C" {

int ustat_plan(const ustat_graph *graph, const ustat_options *opts, ustat_plan_t **out) {
    if (!graph || !opts || !out) return USTAT_ERR_INVALID_ARG;
    ustat_plan_t *p = new (std::nothrow) ustat_plan_t();
    if (!p) return USTAT_ERR_INVALID_ARG;
    int rc = build_plan_best(graph, opts, &p->p);
    if (rc != USTAT_OK) {
        delete p;
        return rc;
    }
    if ((int)p->p.parts.size() > kCombineMaxParts) {
        delete p;
        return USTAT_ERR_UNSUPPORTED;
    }
    *out = p;
    return USTAT_OK;
}

void ustat_plan_destroy(ustat_plan_t *plan) { delete plan; }

namespace {
// Modelled cost of a lowered program at sample size n: each operation's
// algorithmic flops, and at least one n^2 pass per operation.
double shard_cost(const Plan &P, int64_t n) {
    const double dn = (double)n;
    double c = 0.0;
    for (auto &op : P.ops) c += std::max(op.coef * std::pow(dn, op.npow), dn * dn);
    return c;
}
}  // namespace

int ustat_plan_shard(const ustat_graph *graph, const ustat_options *opts, int shard, int n_shards, int64_t n,
                     int *owner, ustat_plan_t **out) {
    if (!graph || !opts || !out || n_shards < 1 || shard < 0 || shard >= n_shards || n < 1)
        return USTAT_ERR_INVALID_ARG;
    Plan full;
    int rc = build_plan_best(graph, opts, &full);
    if (rc != USTAT_OK) return rc;
    const int np = (int)full.parts.size();
    if (np > kCombineMaxParts) return USTAT_ERR_UNSUPPORTED;
    // Groups: evaluated partitions that share a scalar (the same contraction,
    // computed once under sharing) stay on one shard.
    std::vector<int> root(np);
    for (int i = 0; i < np; ++i) root[i] = i;
    auto find = [&](int i) {
        while (root[i] != i) i = root[i] = root[root[i]];
        return i;
    };
    std::vector<int> first_user(full.slots.size(), -1);
    for (int i = 0; i < np; ++i) {
        const PartRec &pr = full.parts[i];
        if (!pr.evaluated) continue;
        for (int q = 0; q < pr.nscal; ++q) {
            int &f = first_user[pr.scal[q]];
            if (f < 0) f = i;
            else root[find(i)] = find(f);
        }
    }
    std::vector<std::vector<int>> groups;
    std::vector<int> group_of(np, -1);
    for (int i = 0; i < np; ++i) {
        if (!full.parts[i].evaluated) continue;
        int r = find(i);
        if (group_of[r] < 0) {
            group_of[r] = (int)groups.size();
            groups.push_back({});
        }
        group_of[i] = group_of[r];
        groups[group_of[i]].push_back(i);
    }
    // Cost of a set of groups: the program that evaluates that set alone, each
    // partition lowered along the elimination order the full plan chose for it
    // (the shards compute the full plan's products); with many partitions (m = 7:
    // 877) groups without an n^3 product skip the estimate.
    const bool many = np > 256;
    std::vector<std::vector<int>> forced(np);
    for (int i = 0; i < np; ++i)
        if (full.parts[i].evaluated)
            forced[i].assign(full.parts[i].order, full.parts[i].order + full.parts[i].nblocks);
    auto cost_of = [&](const std::vector<char> &keep, double *c) {
        PlanRequest req;
        req.keep = &keep;
        req.forced = &forced;
        Plan gp;
        int e = build_plan(graph, opts, &gp, &req);
        *c = e == USTAT_OK ? shard_cost(gp, n) : 0.0;
        return e;
    };
    std::vector<double> cost(groups.size(), 0.0);
    std::vector<int> shard_of_group(groups.size(), 0);
    if (n_shards > 1) {
        for (size_t gi = 0; gi < groups.size(); ++gi) {
            std::vector<char> keep(np, 0);
            for (int i : groups[gi]) keep[i] = 1;
            rc = cost_of(keep, &cost[gi]);
            if (rc != USTAT_OK) return rc;
        }
        // Costliest group first, to the shard that minimises the largest shard
        // cost plus the work the group adds there: a group whose products a
        // shard already computes adds only its own passes, so sharing is kept
        // unless splitting it shortens the longest shard by more than the work
        // it repeats; independent groups go to the least loaded shard.  Ties:
        // the smaller growth, the lower shard.
        std::vector<int> by_cost(groups.size());
        for (size_t gi = 0; gi < groups.size(); ++gi) by_cost[gi] = (int)gi;
        std::stable_sort(by_cost.begin(), by_cost.end(), [&](int a, int b) { return cost[a] > cost[b]; });
        std::vector<std::vector<char>> keep_of(n_shards, std::vector<char>(np, 0));
        std::vector<double> load(n_shards, 0.0);
        double span = 0.0;
        const double dn = (double)n;
        for (int gi : by_cost) {
            if (many && cost[gi] < dn * dn * dn) {
                // no n^3 product: its n^2 passes go to the least loaded shard
                int r = (int)(std::min_element(load.begin(), load.end()) - load.begin());
                shard_of_group[gi] = r;
                load[r] += cost[gi];
                span = std::max(span, load[r]);
                for (int i : groups[gi]) keep_of[r][i] = 1;
                continue;
            }
            int best = -1;
            double best_load = 0.0, best_growth = 0.0, best_score = 0.0;
            for (int r = 0; r < n_shards; ++r) {
                double c = cost[gi];
                if (load[r] > 0.0) {
                    std::vector<char> k = keep_of[r];
                    for (int i : groups[gi]) k[i] = 1;
                    rc = cost_of(k, &c);
                    if (rc != USTAT_OK) return rc;
                }
                double growth = c - load[r];
                double score = std::max(span, c) + growth;
                if (best < 0 || score < best_score || (score == best_score && growth < best_growth)) {
                    best = r;
                    best_load = c;
                    best_growth = growth;
                    best_score = score;
                }
                if (load[r] == 0.0) break;   // empty shards are alike: try the first only
            }
            shard_of_group[gi] = best;
            load[best] = best_load;
            span = std::max(span, best_load);
            for (int i : groups[gi]) keep_of[best][i] = 1;
        }
    }
    std::vector<char> keep(np, 0);
    for (int i = 0; i < np; ++i) {
        int r = group_of[i] < 0 ? -1 : shard_of_group[group_of[i]];
        if (owner) owner[i] = r;
        keep[i] = r == shard;
    }
    ustat_plan_t *p = new (std::nothrow) ustat_plan_t();
    if (!p) return USTAT_ERR_INVALID_ARG;
    PlanRequest req;
    req.keep = &keep;
    req.forced = &forced;
    rc = build_plan(graph, opts, &p->p, &req);
    if (rc != USTAT_OK) {
        delete p;
        return rc;
    }
    *out = p;
    return USTAT_OK;
}

}  // extern "C"

namespace {
// Plan serialisation: a header that names the format and the sizes of the
// records it copies (so a plan written by a build with other record layouts is
// refused), the scalar fields, then each vector as a count and its records.
constexpr uint32_t kPlanMagic = 0x50545355u;   // "USTP"
constexpr uint32_t kPlanFormat = 1;
static_assert(std::is_trivially_copyable<Op>::value && std::is_trivially_copyable<Slot>::value &&
                  std::is_trivially_copyable<PartRec>::value,
              "plan records are copied byte for byte");

struct Writer {
    std::vector<char> b;
    template <typename T> void put(const T &v) {
        const char *p = (const char *)&v;
        b.insert(b.end(), p, p + sizeof(T));
    }
    template <typename T> void vec(const std::vector<T> &v) {
        put<uint64_t>(v.size());
        const char *p = (const char *)v.data();
        b.insert(b.end(), p, p + sizeof(T) * v.size());
    }
};

struct Reader {
    const char *p;
    size_t left;
    bool ok = true;
    template <typename T> T get() {
        T v{};
        if (left < sizeof(T)) {
            ok = false;
            return v;
        }
        std::memcpy(&v, p, sizeof(T));
        p += sizeof(T);
        left -= sizeof(T);
        return v;
    }
    template <typename T> void vec(std::vector<T> &v) {
        uint64_t n = get<uint64_t>();
        if (!ok || n > left / (sizeof(T) ? sizeof(T) : 1)) {
            ok = false;
            return;
        }
        v.resize(n);
        std::memcpy(v.data(), p, sizeof(T) * n);
        p += sizeof(T) * n;
        left -= sizeof(T) * n;
    }
};

void write_plan(const Plan &P, Writer &w) {
    w.put(kPlanMagic);
    w.put(kPlanFormat);
    w.put<uint32_t>(sizeof(Op));
    w.put<uint32_t>(sizeof(Slot));
    w.put<uint32_t>(sizeof(PartRec));
    w.put<int32_t>(P.m);
    w.put<int32_t>(P.precision);
    w.put<int32_t>(P.sparsify);
    w.put<int32_t>(P.planner);
    w.put<int32_t>(P.cse);
    w.put<int32_t>(P.n_gemm);
    w.put<int32_t>(P.n_gemm3);
    for (int c = 0; c < 4; ++c) w.put<int32_t>(P.tc_variant[c]);
    w.vec(P.factor_kind);
    w.vec(P.slots);
    w.vec(P.ops);
    w.vec(P.parts);
    w.put<uint64_t>(P.groups.size());
    for (auto &g : P.groups) w.vec(g);
}
}  // namespace

extern "C" {

int ustat_plan_serialize(const ustat_plan_t *plan, void *buf, size_t buf_len, size_t *needed) {
    if (!plan) return USTAT_ERR_INVALID_ARG;
    Writer w;
    write_plan(plan->p, w);
    if (needed) *needed = w.b.size();
    if (!buf) return USTAT_OK;
    if (buf_len < w.b.size()) return USTAT_ERR_INVALID_ARG;
    std::memcpy(buf, w.b.data(), w.b.size());
    return USTAT_OK;
}

int ustat_plan_deserialize(const void *buf, size_t len, ustat_plan_t **out) {
    if (!buf || !out) return USTAT_ERR_INVALID_ARG;
    Reader r{(const char *)buf, len};
    if (r.get<uint32_t>() != kPlanMagic || r.get<uint32_t>() != kPlanFormat || r.get<uint32_t>() != sizeof(Op) ||
        r.get<uint32_t>() != sizeof(Slot) || r.get<uint32_t>() != sizeof(PartRec) || !r.ok)
        return USTAT_ERR_INVALID_ARG;
    ustat_plan_t *p = new (std::nothrow) ustat_plan_t();
    if (!p) return USTAT_ERR_INVALID_ARG;
    Plan &P = p->p;
    P.m = r.get<int32_t>();
    P.precision = r.get<int32_t>();
    P.sparsify = r.get<int32_t>();
    P.planner = r.get<int32_t>();
    P.cse = r.get<int32_t>();
    P.n_gemm = r.get<int32_t>();
    P.n_gemm3 = r.get<int32_t>();
    for (int c = 0; c < 4; ++c) P.tc_variant[c] = r.get<int32_t>();
    r.vec(P.factor_kind);
    r.vec(P.slots);
    r.vec(P.ops);
    r.vec(P.parts);
    uint64_t ng = r.get<uint64_t>();
    if (r.ok && ng <= r.left) {
        P.groups.resize(ng);
        for (auto &g : P.groups) r.vec(g);
    } else {
        r.ok = false;
    }
    // every record must refer to what the plan holds
    bool valid = r.ok && r.left == 0 && P.m >= 1 && P.m <= kMaxM && P.precision >= USTAT_FP64 &&
                 P.precision <= USTAT_BF16X5 && (int)P.parts.size() <= kCombineMaxParts;
    const int nslots = (int)P.slots.size(), nf = (int)P.factor_kind.size();
    auto slot_ok = [&](int s) { return s >= -1 && s < nslots; };
    auto term_ok = [&](const Term &t) { return slot_ok(t.mat); };
    auto op_ok = [&](const Op &o) {
        bool ok = o.kind >= 0 && o.kind < OP_COUNT && slot_ok(o.out) && o.factor >= -1 && o.factor < nf &&
                  o.nt >= 0 && o.nt <= kMaxTerms && o.nred >= 0 && o.nred <= kMaxRed && slot_ok(o.u) &&
                  slot_ok(o.a) && slot_ok(o.b) && term_ok(o.A) && term_ok(o.B) && term_ok(o.W) && slot_ok(o.opA) &&
                  slot_ok(o.opB) && term_ok(o.Ab) && term_ok(o.Wbc) && term_ok(o.Wbd) && slot_ok(o.ub) &&
                  o.group >= -1 && o.group < (int)P.groups.size();
        for (int t = 0; t < kMaxTerms; ++t) ok = ok && term_ok(o.t[t]);
        for (int q = 0; q < kMaxRed; ++q) ok = ok && term_ok(o.red[q].W) && slot_ok(o.red[q].out) &&
                                                slot_ok(o.red[q].a) && slot_ok(o.red[q].b);
        return ok;
    };
    for (size_t i = 0; valid && i < P.ops.size(); ++i) valid = op_ok(P.ops[i]);
    for (size_t g = 0; valid && g < P.groups.size(); ++g)
        for (auto &o : P.groups[g]) valid = valid && op_ok(o);
    for (size_t i = 0; valid && i < P.parts.size(); ++i) {
        const PartRec &pr = P.parts[i];
        valid = pr.nscal >= 0 && pr.nscal <= kMaxScal;
        for (int q = 0; valid && q < pr.nscal; ++q) valid = pr.scal[q] >= 0 && pr.scal[q] < nslots;
    }
    for (int k : P.factor_kind) valid = valid && k >= USTAT_RBF && k <= USTAT_GRAM;
    if (!valid) {
        delete p;
        return USTAT_ERR_INVALID_ARG;
    }
    *out = p;
    return USTAT_OK;
}

int ustat_plan_info(const ustat_plan_t *plan, int *n_parts, int *mu, int *tw, int *rgs, int *evaluated, int *n_ops,
                    int *n_gemm, int *n_gemm3) {
    if (!plan) return USTAT_ERR_INVALID_ARG;
    const Plan &P = plan->p;
    if (n_parts) *n_parts = (int)P.parts.size();
    for (size_t i = 0; i < P.parts.size(); ++i) {
        if (mu) mu[i] = P.parts[i].mu;
        if (tw) tw[i] = P.parts[i].tw;
        if (evaluated) evaluated[i] = P.parts[i].evaluated;
        if (rgs)
            for (int q = 0; q < P.m; ++q) rgs[i * P.m + q] = P.parts[i].rgs[q];
    }
    if (n_ops) *n_ops = (int)P.ops.size();
    if (n_gemm) *n_gemm = P.n_gemm;
    if (n_gemm3) *n_gemm3 = P.n_gemm3;
    return USTAT_OK;
}

int ustat_plan_flops(const ustat_plan_t *plan, int64_t n, double *flops_plan, double *flops_naive) {
    if (!plan || n < 1) return USTAT_ERR_INVALID_ARG;
    const Plan &P = plan->p;
    const double dn = (double)n;
    double fp = 0.0, fn = 0.0;
    for (auto &op : P.ops) fp += op.coef * std::pow(dn, op.npow);
    for (auto &pr : P.parts)
        if (pr.evaluated)
            for (int q = 0; q < 5; ++q) fn += pr.naive_coef[q] * std::pow(dn, q + 1);
    if (flops_plan) *flops_plan = fp;
    if (flops_naive) *flops_naive = fn;
    return USTAT_OK;
}

int ustat_status(const void *ws, void *stream, int *device_status) {
    if (!ws || !device_status) return USTAT_ERR_INVALID_ARG;
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e);
    int word = 0;   // every workspace layout starts with the error word (Layout::err_off = 0)
    e = cudaMemcpy(&word, ws, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e);
    *device_status = status_of_word(word);
    return USTAT_OK;
}

int ustat_factor_matrix(int kind, double param, const double *data, int64_t n, double *F, void *ws,
                        void *stream) {
    if (!data || !F || !ws || n < 1 || ((uintptr_t)ws & 255)) return USTAT_ERR_INVALID_ARG;
    if (n > (int64_t)1 << 20) return USTAT_ERR_UNSUPPORTED;
    const bool pairs = kind == USTAT_DIST || kind == USTAT_LOWRANK || kind == USTAT_GRAM;
    if (!pairs && kind != USTAT_COMPLEMENT) return USTAT_ERR_INVALID_ARG;
    if (pairs && !(param >= 1.0 && param <= 4096.0 && param == (double)(int)param)) return USTAT_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int *err = (int *)ws;   // the error word, at offset 0 as in every evaluation workspace
    cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), st);
    if (e == cudaSuccess)
        e = pairs ? launch_pairs(kind, data, (int)param, n, true, 0, F, err, st)
                  : launch_loadmat(data, n, true, 0, 1, F, err, st);
    return e == cudaSuccess ? USTAT_OK : cuda_fail(e);
}

int ustat_workspace_bytes(const ustat_plan_t *plan, int64_t n, int d, size_t *bytes) {
    if (!plan || !bytes || n < 1 || d < 1) return USTAT_ERR_INVALID_ARG;
    *bytes = make_layout(plan->p, n, d).total;
    return USTAT_OK;
}

int ustat_eval(ustat_plan_t *plan, const void *X, int x_dtype, int64_t n, int d, const ustat_factor *factors,
               int n_factors, void *ws, size_t ws_bytes, void *stream, double *U_out, double *V_out) {
    if (!plan || !X || !U_out || d < 1 || n < 1 || (x_dtype != 0 && x_dtype != 1)) return USTAT_ERR_INVALID_ARG;
    const Plan &P = plan->p;
    if (n < P.m) return USTAT_ERR_N_LT_M;
    if (n > (int64_t)1 << 20) return USTAT_ERR_UNSUPPORTED;
    int rc = check_graph_factors(P, factors, n_factors, d);
    if (rc != USTAT_OK) return rc;
    Layout L = make_layout(P, n, d);
    if (!ws || ws_bytes < L.total || ((uintptr_t)ws % 256) != 0) return USTAT_ERR_WORKSPACE;
    Ctx C{P, L, (char *)ws, n, d, wide_storage(P.precision), (cudaStream_t)stream};
    return run_program(C, X, x_dtype, factors, U_out, V_out);
}

int ustat_scalar_count(const ustat_plan_t *plan, int *count) {
    if (!plan || !count) return USTAT_ERR_INVALID_ARG;
    int ns = 0;
    for (auto &sl : plan->p.slots) ns += sl.kind == S_SCAL;
    *count = ns;
    return USTAT_OK;
}

int ustat_eval_rows(ustat_plan_t *plan, int rank, int n_ranks, const void *X, int x_dtype, int64_t n, int d,
                    const ustat_factor *factors, int n_factors, void *ws, size_t ws_bytes, void *stream,
                    double *scal_out) {
    if (!plan || !X || !scal_out || d < 1 || n < 1 || (x_dtype != 0 && x_dtype != 1) || n_ranks < 1 || rank < 0 ||
        rank >= n_ranks)
        return USTAT_ERR_INVALID_ARG;
    const Plan &P = plan->p;
    if (n < P.m) return USTAT_ERR_N_LT_M;
    if (n > (int64_t)1 << 20) return USTAT_ERR_UNSUPPORTED;
    std::vector<char> sharded;
    if (!row_shard_slots(P, sharded)) return USTAT_ERR_UNSUPPORTED;
    int rc = check_graph_factors(P, factors, n_factors, d);
    if (rc != USTAT_OK) return rc;
    Layout L = make_layout(P, n, d);
    if (!ws || ws_bytes < L.total || ((uintptr_t)ws % 256) != 0) return USTAT_ERR_WORKSPACE;
    Ctx C{P, L, (char *)ws, n, d, wide_storage(P.precision), (cudaStream_t)stream};
    C.rank = rank;
    C.nranks = n_ranks;
    return run_program(C, X, x_dtype, factors, nullptr, nullptr, scal_out);
}

int ustat_lean_workspace_bytes(const ustat_plan_t *plan, int64_t n, int d, int64_t panel_rows, size_t *bytes) {
    if (!plan || !bytes || n < 1 || d < 1 || panel_rows < 128 || panel_rows % 128 != 0) return USTAT_ERR_INVALID_ARG;
    const LeanPlan LP = lean_plan(plan->p);
    if (!LP.ok || d > 256) return USTAT_ERR_UNSUPPORTED;
    *bytes = make_lean_layout(plan->p, n, d, std::min<int64_t>(panel_rows, align_up((size_t)n, 128)), LP.need_k)
                 .L.total;
    return USTAT_OK;
}

int ustat_eval_lean(ustat_plan_t *plan, const void *X, int x_dtype, int64_t n, int d, const ustat_factor *factors,
                    int n_factors, int64_t panel_rows, void *ws, size_t ws_bytes, void *stream, double *U_out,
                    double *V_out) {
    if (!plan || !X || !U_out || d < 1 || n < 1 || (x_dtype != 0 && x_dtype != 1) || panel_rows < 128 ||
        panel_rows % 128 != 0)
        return USTAT_ERR_INVALID_ARG;
    const Plan &P = plan->p;
    if (n < P.m) return USTAT_ERR_N_LT_M;
    if (n > (int64_t)1 << 20) return USTAT_ERR_UNSUPPORTED;
    const LeanPlan LP = lean_plan(P);
    if (!LP.ok || d > 256) return USTAT_ERR_UNSUPPORTED;
    int rc = check_graph_factors(P, factors, n_factors, d);
    if (rc != USTAT_OK) return rc;
    const int64_t panel = std::min<int64_t>(panel_rows, align_up((size_t)n, 128));
    LeanLayout LL = make_lean_layout(P, n, d, panel, LP.need_k);
    if (!ws || ws_bytes < LL.L.total || ((uintptr_t)ws % 256) != 0) return USTAT_ERR_WORKSPACE;
    return run_lean(P, LP, LL, (char *)ws, n, d, panel, X, x_dtype, factors, (cudaStream_t)stream, U_out, V_out);
}

int ustat_combine(const ustat_plan_t *plan, const double *scal, int64_t n, void *stream, double *U_out,
                  double *V_out) {
    if (!plan || !scal || !U_out || n < 1) return USTAT_ERR_INVALID_ARG;
    const Plan &P = plan->p;
    if (n < P.m) return USTAT_ERR_N_LT_M;
    Layout L = make_layout(P, n, 1);
    cudaError_t e = plan_combine(P, L, scal, nullptr, n, U_out, V_out, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e);
    return USTAT_OK;
}

int ustat_host_staging_bytes(const ustat_plan_t *plan, int64_t n, int d, size_t *bytes) {
    if (!plan || !bytes || n < 1 || d < 1) return USTAT_ERR_INVALID_ARG;
    *bytes = align_up(8 * (size_t)n * d, 1024) + align_up(8 * (2 + plan->p.parts.size()), 1024);
    return USTAT_OK;
}

int ustat_eval_host(ustat_plan_t *plan, const void *X_host, int x_dtype, int64_t n, int d,
                    const ustat_factor *factors, int n_factors, void *ws, size_t ws_bytes, void *stream,
                    double *U_host, double *V_host) {
    if (!plan || !X_host || !U_host || d < 1 || n < 1 || (x_dtype != 0 && x_dtype != 1)) return USTAT_ERR_INVALID_ARG;
    const Plan &P = plan->p;
    if (n < P.m) return USTAT_ERR_N_LT_M;
    size_t main_bytes = make_layout(P, n, d).total, stage = 0;
    ustat_host_staging_bytes(plan, n, d, &stage);
    if (!ws || ws_bytes < main_bytes + stage) return USTAT_ERR_WORKSPACE;
    char *xs = (char *)ws + main_bytes;
    double *outs = (double *)(xs + align_up(8 * (size_t)n * d, 1024));
    cudaStream_t st = (cudaStream_t)stream;
    const size_t xbytes = (x_dtype == 0 ? 8 : 4) * (size_t)n * d;
    cudaError_t e = cudaMemcpyAsync(xs, X_host, xbytes, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e);
    int rc = ustat_eval(plan, xs, x_dtype, n, d, factors, n_factors, ws, main_bytes, stream, outs, outs + 2);
    if (rc != USTAT_OK) return rc;
    e = cudaMemcpyAsync(U_host, outs, 2 * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && V_host)
        e = cudaMemcpyAsync(V_host, outs + 2, P.parts.size() * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail(e);
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e);
    return USTAT_OK;
}

int ustat_batch_workspace_bytes(const ustat_plan_t *plan, const int64_t *n, int count, int d, size_t *bytes) {
    if (!plan || !n || count < 1 || !bytes) return USTAT_ERR_INVALID_ARG;
    int64_t mx = 0;
    for (int i = 0; i < count; ++i) mx = std::max(mx, n[i]);
    return ustat_workspace_bytes(plan, mx, d, bytes);
}

int ustat_eval_batch(ustat_plan_t *plan, const void *const *X, int x_dtype, const int64_t *n, int count, int d,
                     const ustat_factor *factors, int n_factors, void *ws, size_t ws_bytes, void *stream,
                     double *U_out, double *V_out) {
    if (!plan || !X || !n || count < 1 || !U_out) return USTAT_ERR_INVALID_ARG;
    const int np = (int)plan->p.parts.size();
    for (int i = 0; i < count; ++i) {
        int rc = ustat_eval(plan, X[i], x_dtype, n[i], d, factors, n_factors, ws, ws_bytes, stream, U_out + 2 * i,
                            V_out ? V_out + (size_t)i * np : nullptr);
        if (rc != USTAT_OK) return rc;
    }
    return USTAT_OK;
}

int ustat_debug_set_wait(long long limit_cycles, int stall_producer) {
    if (limit_cycles < 0) return USTAT_ERR_INVALID_ARG;
    set_tc_debug(limit_cycles, stall_producer);
    return USTAT_OK;
}

int ustat_profile_enable(int enable) {
    g_prof.on = enable != 0;
    return USTAT_OK;
}

int ustat_profile_kinds(void) { return kProfKinds; }

const char *ustat_profile_kind_name(int kind) {
    if (kind == kProfXconvert) return "xconvert";
    if (kind == kProfCombine) return "combine";
    return op_name(kind);
}

int ustat_profile_collect(double *ms, int *launches) {
    for (auto &r : g_prof.recs) {
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e != cudaSuccess) return cuda_fail(e);
        float t = 0.f;
        e = cudaEventElapsedTime(&t, r.a, r.b);
        if (e != cudaSuccess) return cuda_fail(e);
        if (ms) ms[r.kind] += t;
        if (launches) launches[r.kind] += r.kernels;
    }
    g_prof.recs.clear();
    g_prof.used = 0;
    return USTAT_OK;
}

const char *ustat_last_cuda_error(void) { return g_last_cuda_error.c_str(); }

const char *ustat_strerror(int code) {
    switch (code) {
        case USTAT_OK: return "ok";
        case USTAT_ERR_INVALID_ARG: return "invalid argument";
        case USTAT_ERR_N_LT_M: return "sample size n is smaller than the order m";
        case USTAT_ERR_TW_TOO_LARGE: return "no executable elimination order (treewidth too large)";
        case USTAT_ERR_WORKSPACE: return "workspace missing, too small or misaligned";
        case USTAT_ERR_NONFINITE: return "non-finite input";
        case USTAT_ERR_CUDA: return "CUDA error";
        case USTAT_ERR_DEVICE_TIMEOUT: return "bounded device wait ran out";
        case USTAT_ERR_UNSUPPORTED: return "unsupported";
        default: return "unknown error";
    }
}

const char *ustat_version(void) { return "ustat-gb300 0.1"; }

}  // extern "C"

extern "C" int ustat_plan_describe(const ustat_plan_t *plan, char *buf, size_t buf_len, size_t *needed) {
    if (!plan) return USTAT_ERR_INVALID_ARG;
    const Plan &P = plan->p;
    std::string s;
    char line[512];
    auto term = [&](const Term &t) -> std::string {
        if (t.mat < 0) return "1";
        return "M" + std::to_string(t.mat) + (t.trans ? "^T" : "");
    };
    auto vec = [&](int v) -> std::string { return v < 0 ? "1" : "v" + std::to_string(v); };
    for (size_t i = 0; i < P.ops.size(); ++i) {
        const Op &o = P.ops[i];
        std::string ts, rs;
        for (int t = 0; t < o.nt; ++t) ts += (t ? "," : "") + term(o.t[t]);
        for (int r = 0; r < o.nred; ++r)
            rs += (r ? ";" : "") + std::string("s") + std::to_string(o.red[r].out) + "+=C^" +
                  std::to_string(o.red[r].pow) + "*" + term(o.red[r].W) + "*" + vec(o.red[r].a) + "*" +
                  vec(o.red[r].b);
        if (o.kind == OP_GEMM) {
            snprintf(line, sizeof(line), "%zu gemm store=%d out=%d A=%s B=%s u=%s sym=%d opA=%d opB=%d red=[%s]\n", i,
                     o.store, o.out, term(o.A).c_str(), term(o.B).c_str(), vec(o.u).c_str(), o.symmetric, o.opA,
                     o.opB, rs.c_str());
        } else if (o.kind == OP_MHB) {
            std::string ms;
            for (const Op &m : P.groups[o.group]) {
                std::string mt;
                for (int t = 0; t < m.nt; ++t) mt += (t ? "," : "") + term(m.t[t]);
                ms += std::string(" ") + op_name(m.kind) + "(out=" + std::to_string(m.out) + " [" + mt + "] " +
                      (m.kind == OP_GEMV ? "u=" + vec(m.u) : "a=" + vec(m.a) + " b=" + vec(m.b)) + ")";
            }
            snprintf(line, sizeof(line), "%zu mhb%s\n", i, ms.c_str());
        } else if (o.kind == OP_KBUILD) {
            std::string ks;
            for (int r = 0; r < o.nred; ++r)
                ks += (r ? ";" : "") + std::string(P.slots[o.red[r].out].kind == S_VEC ? "v" : "s") +
                      std::to_string(o.red[r].out) + "+=K^" + std::to_string(o.red[r].pow);
            snprintf(line, sizeof(line), "%zu kbuild out=%d f=%d slices=%d upper=%d red=[%s]\n", i, o.out, o.factor,
                     o.opA, o.upper_only, ks.c_str());
        }
        else
            snprintf(line, sizeof(line),
                     "%zu %s out=%d f=%d terms=[%s] u=%s a=%s b=%s A=%s B=%s W=%s Ab=%s Wbc=%s Wbd=%s ub=%s\n", i,
                     op_name(o.kind), o.out, o.factor, ts.c_str(), vec(o.u).c_str(), vec(o.a).c_str(),
                     vec(o.b).c_str(), term(o.A).c_str(), term(o.B).c_str(), term(o.W).c_str(), term(o.Ab).c_str(),
                     term(o.Wbc).c_str(), term(o.Wbd).c_str(), vec(o.ub).c_str());
        s += line;
    }
    snprintf(line, sizeof(line), "tc_variant=[%d,%d,%d,%d]\n", P.tc_variant[0], P.tc_variant[1], P.tc_variant[2],
             P.tc_variant[3]);
    s += line;
    for (size_t p = 0; p < P.parts.size(); ++p) {
        const PartRec &r = P.parts[p];
        std::string rg, sc;
        for (int q = 0; q < P.m; ++q) rg += std::to_string(r.rgs[q]);
        for (int q = 0; q < r.nscal; ++q) sc += (q ? "," : "") + std::to_string(r.scal[q]);
        snprintf(line, sizeof(line), "part %zu rgs=%s mu=%d tw=%d eval=%d nfree=%d scal=[%s]\n", p, rg.c_str(), r.mu,
                 r.tw, r.evaluated, r.nfree, sc.c_str());
        s += line;
    }
    if (needed) *needed = s.size() + 1;
    if (buf && buf_len) {
        size_t k = std::min(buf_len - 1, s.size());
        std::memcpy(buf, s.data(), k);
        buf[k] = 0;
    }
    return USTAT_OK;
}

// ---------------------------------------------------------------- no-allocation entry point
// Scratch used in place of a caller workspace by ustat_eval_noalloc, for callers
// that may not allocate device memory at evaluation time (a service that reserves
// its memory at start-up, a plug-in inside another framework's allocator, a
// latency-critical path where cudaMalloc may stall or synchronise).  In host
// code the name below is a host-side stand-in, not a device address: the
// device address is looked up per device with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[USTAT_NOALLOC_MAX_BYTES];

namespace {
constexpr int kNoallocMaxDevices = 64;
void *g_noalloc_addr[kNoallocMaxDevices] = {nullptr};
std::mutex g_noalloc_mu;
}  // namespace

extern "C" int ustat_eval_noalloc(ustat_plan_t *plan, const void *X, int x_dtype, int64_t n, int d,
                                  const ustat_factor *factors, int n_factors, void *stream, double *U_out,
                                  double *V_out) {
    if (!plan || !X || !U_out || d < 1 || n < 1 || (x_dtype != 0 && x_dtype != 1)) return USTAT_ERR_INVALID_ARG;
    size_t need = 0;
    int rc = ustat_workspace_bytes(plan, n, d, &need);
    if (rc != USTAT_OK) return rc;
    if (need > (size_t)USTAT_NOALLOC_MAX_BYTES) return USTAT_ERR_WORKSPACE;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e);
    if (dev < 0 || dev >= kNoallocMaxDevices) return USTAT_ERR_UNSUPPORTED;
    void *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_addr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) return cuda_fail(e);
            g_noalloc_addr[dev] = p;
        }
        base = g_noalloc_addr[dev];
    }
    return ustat_eval(plan, X, x_dtype, n, d, factors, n_factors, base, (size_t)USTAT_NOALLOC_MAX_BYTES, stream, U_out,
                      V_out);
}

extern "C" int ustat_noalloc_status(void *stream, int *device_status) {
    if (!device_status) return USTAT_ERR_INVALID_ARG;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e);
    if (dev < 0 || dev >= kNoallocMaxDevices) return USTAT_ERR_UNSUPPORTED;
    void *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        base = g_noalloc_addr[dev];
    }
    if (!base) {
        // no evaluation on this device yet: nothing can have failed
        *device_status = USTAT_OK;
        return USTAT_OK;
    }
    return ustat_status(base, stream, device_status);
}

// ---------------------------------------------------------------- batched evaluation
// Samples spread over CUDA streams ("lanes") by longest-processing-time first,
// each lane with its own workspace region; the lanes fork from and join into
// the caller's stream.  A whole batch can be captured into one CUDA graph.
struct ustat_batched {
    ustat_plan_t *plan = nullptr;
    int d = 0;
    std::vector<int64_t> n;
    int max_lanes = 1, lanes = 1;
    std::vector<int> lane_of;
    size_t lane_bytes = 0;
    int device = -1;
    std::vector<cudaStream_t> streams;   // max_lanes, created at the first run
    std::vector<cudaEvent_t> joins;
    cudaEvent_t fork = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    // grouped form (ustat_batched_set_grouped): one workspace region per sample, the
    // plan run step by step over all samples, every bf16x3 product step as one
    // persistent launch over all samples' tiles
    int grouped = 0;
    std::vector<size_t> soff;                 // per sample: its region's offset
    std::vector<size_t> goff;                 // per product step: its group image's offset
    size_t grouped_bytes = 0;
    std::vector<std::vector<char>> images;    // host copies of the group images
    std::vector<int> image_tiles, image_shape;
    const void *image_ws = nullptr;
    int image_var[4] = {-1, -1, -1, -1};
};

namespace {

void batched_schedule(ustat_batched *b) {
    const Plan &P = b->plan->p;
    const int cnt = (int)b->n.size();
    std::vector<int> order(cnt);
    std::vector<double> cost(cnt);
    for (int i = 0; i < cnt; ++i) {
        double fp = 0.0;
        for (auto &op : P.ops) fp += op.coef * std::pow((double)b->n[i], op.npow);
        // a fixed per-sample charge for the launches of small samples
        cost[i] = fp + 2.0e9;
        order[i] = i;
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return cost[a] > cost[c]; });
    std::vector<double> load(b->lanes, 0.0);
    b->lane_of.assign(cnt, 0);
    for (int i : order) {
        int best = 0;
        for (int l = 1; l < b->lanes; ++l)
            if (load[l] < load[best]) best = l;
        b->lane_of[i] = best;
        load[best] += cost[i];
    }
}

// the product steps that run as one grouped launch in the grouped form
bool group_step(const Plan &P, const Op &op) { return P.precision == USTAT_BF16X3 && op.kind == OP_GEMM; }

void batched_grouped_layout(ustat_batched *b) {
    const Plan &P = b->plan->p;
    size_t cur = 0;
    b->soff.assign(b->n.size(), 0);
    for (size_t i = 0; i < b->n.size(); ++i) {
        b->soff[i] = cur;
        cur = align_up(cur + make_layout(P, b->n[i], b->d).total, 1024);
    }
    b->goff.clear();
    for (const Op &op : P.ops)
        if (group_step(P, op)) {
            b->goff.push_back(cur);
            cur = align_up(cur + gemm_group_bytes((int)b->n.size()), 1024);
        }
    b->grouped_bytes = cur;
    b->image_ws = nullptr;
}

size_t batched_ws_bytes(const ustat_batched *b) {
    return b->grouped ? b->grouped_bytes : (size_t)b->max_lanes * b->lane_bytes;
}

// The group images of the product steps for workspace ws: each sample's product
// arguments (its own region), the largest samples first, built on the host and
// copied to the workspace on the stream (before any capture: the copies are not
// part of a graph).  Rebuilt when the workspace or the plan's variants change.
int batched_group_prepare(ustat_batched *b, char *ws, cudaStream_t st) {
    const Plan &P = b->plan->p;
    bool same = b->image_ws == ws;
    for (int c = 0; c < 4; ++c) same = same && b->image_var[c] == P.tc_variant[c];
    if (same) return USTAT_OK;
    const int cnt = (int)b->n.size();
    std::vector<int> order(cnt);
    for (int i = 0; i < cnt; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return b->n[x] > b->n[y]; });
    b->images.clear();
    b->image_tiles.clear();
    b->image_shape.clear();
    size_t k = 0;
    for (const Op &op : P.ops) {
        if (!group_step(P, op)) continue;
        std::vector<TcGemmArgs> items(cnt);
        int shape0 = -1;
        for (int q = 0; q < cnt; ++q) {
            const int i = order[q];
            Layout L = make_layout(P, b->n[i], b->d);
            Ctx C{P, L, ws + b->soff[i], b->n[i], b->d, false, st};
            ProgState S;
            S.err = (int *)(C.ws + L.err_off);
            S.lead = split_lead_bits(b->n[i]);
            S.D = diag_fix_of(P, b->n[i]);
            int shape = 0;
            tc_gemm_args(C, op, S, items[q], shape);
            if (q == 0) shape0 = shape;   // the largest sample's size class picks the tile shape
        }
        if (shape0 == 1 && op.symmetric) shape0 = 0;
        std::vector<char> host;
        const int tiles = gemm_group_image(items.data(), cnt, shape0, ws + b->goff[k], host);
        if (tiles < 0) return USTAT_ERR_UNSUPPORTED;
        cudaError_t e = cudaMemcpyAsync(ws + b->goff[k], host.data(), host.size(), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e);
        b->images.push_back(std::move(host));
        b->image_tiles.push_back(tiles);
        b->image_shape.push_back(shape0);
        ++k;
    }
    // the pageable host images must outlive their copies
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e);
    b->image_ws = ws;
    for (int c = 0; c < 4; ++c) b->image_var[c] = P.tc_variant[c];
    return USTAT_OK;
}

int batched_setup(ustat_batched *b) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e);
    if (b->device >= 0) return dev == b->device ? USTAT_OK : USTAT_ERR_INVALID_ARG;
    b->streams.assign(b->max_lanes, nullptr);
    b->joins.assign(b->max_lanes, nullptr);
    for (int l = 0; l < b->max_lanes; ++l) {
        e = cudaStreamCreateWithFlags(&b->streams[l], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->joins[l], cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(e);
    b->device = dev;
    return USTAT_OK;
}

// The grouped form: every sample in its own region, the plan step by step; the
// samples' steps on the lanes, each product step one grouped launch on the
// caller's stream between a join of the lanes and a new fork.
int batched_body_grouped(ustat_batched *b, const void *const *X, int x_dtype, const ustat_factor *f, char *ws,
                         cudaStream_t st, double *U_out, double *V_out) {
    const Plan &P = b->plan->p;
    const int np = (int)P.parts.size();
    const int cnt = (int)b->n.size();
    std::vector<Layout> Ls(cnt);
    for (int i = 0; i < cnt; ++i) Ls[i] = make_layout(P, b->n[i], b->d);
    auto ctx = [&](int i) {
        return Ctx{P, Ls[i], ws + b->soff[i], b->n[i], b->d, wide_storage(P.precision), b->streams[b->lane_of[i]]};
    };
    auto fork = [&]() -> cudaError_t {
        cudaError_t e = cudaEventRecord(b->fork, st);
        for (int l = 0; l < b->lanes && e == cudaSuccess; ++l) e = cudaStreamWaitEvent(b->streams[l], b->fork, 0);
        return e;
    };
    auto join = [&]() -> cudaError_t {
        cudaError_t e = cudaSuccess;
        for (int l = 0; l < b->lanes && e == cudaSuccess; ++l) {
            e = cudaEventRecord(b->joins[l], b->streams[l]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(st, b->joins[l], 0);
        }
        return e;
    };
    cudaError_t e = fork();
    if (e != cudaSuccess) return cuda_fail(e);
    std::vector<ProgState> S(cnt);
    for (int i = 0; i < cnt; ++i) {
        int rc = program_prologue(ctx(i), X[i], x_dtype, f, S[i]);
        if (rc != USTAT_OK) return rc;
    }
    size_t k = 0;
    for (const Op &op : P.ops) {
        if (group_step(P, op)) {
            e = join();
            if (e == cudaSuccess) {
                ProfScope ps(op.kind, st);
                e = launch_gemm_group(ws + b->goff[k], cnt, b->image_tiles[k], b->image_shape[k], S[0].err, st);
            }
            if (e == cudaSuccess) e = fork();
            if (e != cudaSuccess) return cuda_fail(e);
            ++k;
            continue;
        }
        for (int i = 0; i < cnt; ++i) {
            int rc = run_op(ctx(i), op, S[i], X[i], x_dtype, f);
            if (rc != USTAT_OK) return rc;
        }
    }
    for (int i = 0; i < cnt && e == cudaSuccess; ++i) {
        const Ctx C = ctx(i);
        ProfScope ps(kProfCombine, C.st);
        e = plan_combine(P, Ls[i], (const double *)(C.ws + Ls[i].scal_off), S[i].err, b->n[i], U_out + 2 * i,
                         V_out ? V_out + (size_t)i * np : nullptr, C.st);
    }
    if (e == cudaSuccess) e = join();
    return e == cudaSuccess ? USTAT_OK : cuda_fail(e);
}

int batched_body(ustat_batched *b, const void *const *X, int x_dtype, const ustat_factor *f, int nf, char *ws,
                 cudaStream_t st, double *U_out, double *V_out) {
    if (b->grouped) return batched_body_grouped(b, X, x_dtype, f, ws, st, U_out, V_out);
    const Plan &P = b->plan->p;
    const int np = (int)P.parts.size();
    cudaError_t e = cudaEventRecord(b->fork, st);
    if (e != cudaSuccess) return cuda_fail(e);
    for (int l = 0; l < b->lanes; ++l) {
        e = cudaStreamWaitEvent(b->streams[l], b->fork, 0);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    for (int l = 0; l < b->lanes; ++l) {
        char *lws = ws + (size_t)l * b->lane_bytes;
        for (size_t i = 0; i < b->n.size(); ++i) {
            if (b->lane_of[i] != l) continue;
            Layout L = make_layout(P, b->n[i], b->d);
            Ctx C{P, L, lws, b->n[i], b->d, wide_storage(P.precision), b->streams[l]};
            int rc = run_program(C, X[i], x_dtype, f, U_out + 2 * i, V_out ? V_out + i * (size_t)np : nullptr);
            if (rc != USTAT_OK) return rc;
        }
    }
    for (int l = 0; l < b->lanes; ++l) {
        e = cudaEventRecord(b->joins[l], b->streams[l]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, b->joins[l], 0);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    return USTAT_OK;
}

int batched_check(ustat_batched *b, const void *const *X, int x_dtype, const ustat_factor *f, int nf, void *ws,
                  size_t ws_bytes, double *U_out) {
    if (!b || !X || !U_out || (x_dtype != 0 && x_dtype != 1)) return USTAT_ERR_INVALID_ARG;
    const Plan &P = b->plan->p;
    int rc = check_graph_factors(P, f, nf, b->d);
    if (rc != USTAT_OK) return rc;
    for (int i = 0; i < nf; ++i)
        if (f[i].kind == USTAT_MATRIX || f[i].kind == USTAT_VECTOR || f[i].kind == USTAT_DIST ||
            f[i].kind == USTAT_LOWRANK || f[i].kind == USTAT_COMPLEMENT || f[i].kind == USTAT_GRAM)
            return USTAT_ERR_UNSUPPORTED;   // data of one size, not per sample
    for (size_t i = 0; i < b->n.size(); ++i)
        if (!X[i]) return USTAT_ERR_INVALID_ARG;
    if (!ws || ((uintptr_t)ws % 256) != 0 || ws_bytes < batched_ws_bytes(b)) return USTAT_ERR_WORKSPACE;
    return batched_setup(b);
}

}  // namespace

extern "C" {

int ustat_plan_set_variant(ustat_plan_t *plan, int size_class, int variant) {
    if (!plan || size_class < -1 || size_class > 3 || variant < 0 || variant > 255 || ((variant >> 2) & 3) == 3)
        return USTAT_ERR_INVALID_ARG;
    for (int c = 0; c < 4; ++c)
        if (size_class < 0 || c == size_class) plan->p.tc_variant[c] = variant;
    return USTAT_OK;
}

int ustat_batched_create(ustat_plan_t *plan, const int64_t *n, int count, int d, int max_lanes,
                         ustat_batched_t **out) {
    if (!plan || !n || count < 1 || d < 1 || !out || max_lanes < 0 || max_lanes > 32) return USTAT_ERR_INVALID_ARG;
    const Plan &P = plan->p;
    for (int i = 0; i < count; ++i) {
        if (n[i] < P.m) return USTAT_ERR_N_LT_M;
        if (n[i] > (int64_t)1 << 20) return USTAT_ERR_UNSUPPORTED;
    }
    ustat_batched *b = new (std::nothrow) ustat_batched();
    if (!b) return USTAT_ERR_INVALID_ARG;
    b->plan = plan;
    b->d = d;
    b->n.assign(n, n + count);
    b->max_lanes = max_lanes == 0 ? 8 : max_lanes;
    b->lanes = std::min(b->max_lanes, count);
    for (int i = 0; i < count; ++i) b->lane_bytes = std::max(b->lane_bytes, make_layout(P, n[i], d).total);
    b->lane_bytes = align_up(b->lane_bytes, 256);
    batched_schedule(b);
    *out = b;
    return USTAT_OK;
}

void ustat_batched_destroy(ustat_batched_t *b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (auto s : b->streams)
        if (s) cudaStreamDestroy(s);
    for (auto e : b->joins)
        if (e) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    delete b;
}

int ustat_batched_workspace_bytes(const ustat_batched_t *b, size_t *bytes) {
    if (!b || !bytes) return USTAT_ERR_INVALID_ARG;
    *bytes = batched_ws_bytes(b);
    return USTAT_OK;
}

int ustat_batched_set_grouped(ustat_batched_t *b, int grouped) {
    if (!b) return USTAT_ERR_INVALID_ARG;
    if (grouped && b->plan->p.precision != USTAT_BF16X3) return USTAT_ERR_UNSUPPORTED;
    b->grouped = grouped != 0;
    if (b->grouped) batched_grouped_layout(b);
    if (b->exec) {   // a captured graph of the other form
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    if (b->graph) {
        cudaGraphDestroy(b->graph);
        b->graph = nullptr;
    }
    return USTAT_OK;
}

int ustat_batched_info(const ustat_batched_t *b, int *lanes, int *lane_of) {
    if (!b) return USTAT_ERR_INVALID_ARG;
    if (lanes) *lanes = b->lanes;
    if (lane_of)
        for (size_t i = 0; i < b->lane_of.size(); ++i) lane_of[i] = b->lane_of[i];
    return USTAT_OK;
}

int ustat_batched_set_lanes(ustat_batched_t *b, int lanes) {
    if (!b || lanes < 1 || lanes > b->max_lanes) return USTAT_ERR_INVALID_ARG;
    b->lanes = std::min(lanes, (int)b->n.size());
    batched_schedule(b);
    return USTAT_OK;
}

int ustat_batched_run(ustat_batched_t *b, const void *const *X, int x_dtype, const ustat_factor *factors,
                      int n_factors, void *ws, size_t ws_bytes, void *stream, double *U_out, double *V_out) {
    int rc = batched_check(b, X, x_dtype, factors, n_factors, ws, ws_bytes, U_out);
    if (rc != USTAT_OK) return rc;
    if (b->grouped && (rc = batched_group_prepare(b, (char *)ws, (cudaStream_t)stream)) != USTAT_OK) return rc;
    return batched_body(b, X, x_dtype, factors, n_factors, (char *)ws, (cudaStream_t)stream, U_out, V_out);
}

int ustat_batched_capture(ustat_batched_t *b, const void *const *X, int x_dtype, const ustat_factor *factors,
                          int n_factors, void *ws, size_t ws_bytes, void *stream, double *U_out, double *V_out) {
    int rc = batched_check(b, X, x_dtype, factors, n_factors, ws, ws_bytes, U_out);
    if (rc != USTAT_OK) return rc;
    if (!stream || g_prof.on) return USTAT_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    if (b->graph) {
        cudaGraphDestroy(b->graph);
        b->graph = nullptr;
    }
    if (b->grouped && (rc = batched_group_prepare(b, (char *)ws, st)) != USTAT_OK) return rc;
    if (tc_gemm3(b->plan->p)) {
        // the treewidth-3 steps' second stream and events, created before the capture
        SideStream *side = nullptr;
        cudaError_t es = side_stream(&side);
        if (es != cudaSuccess) return cuda_fail(es);
    }
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e);
    rc = batched_body(b, X, x_dtype, factors, n_factors, (char *)ws, st, U_out, V_out);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(st, &g);
    if (rc != USTAT_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e);
    b->graph = g;
    e = cudaGraphInstantiate(&b->exec, g, 0);
    if (e != cudaSuccess) return cuda_fail(e);
    return USTAT_OK;
}

int ustat_batched_replay(ustat_batched_t *b, void *stream) {
    if (!b || !b->exec) return USTAT_ERR_INVALID_ARG;
    cudaError_t e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
    return e == cudaSuccess ? USTAT_OK : cuda_fail(e);
}

int ustat_batched_autotune(ustat_batched_t *b, const void *const *X, int x_dtype, const ustat_factor *factors,
                           int n_factors, void *ws, size_t ws_bytes, void *stream, double *U_out, double *V_out,
                           int *lanes_out, double *ms_out) {
    int rc = batched_check(b, X, x_dtype, factors, n_factors, ws, ws_bytes, U_out);
    if (rc != USTAT_OK) return rc;
    if (g_prof.on) return USTAT_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    Plan &P = b->plan->p;
    cudaEvent_t t0, t1;
    cudaError_t e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    if (e != cudaSuccess) return cuda_fail(e);
    // time of one batched evaluation: the best of two after a warm-up
    auto timed = [&](double *ms) -> int {
        if (b->grouped) {   // the group images follow the variants (built outside the timing)
            int r = batched_group_prepare(b, (char *)ws, st);
            if (r != USTAT_OK) return r;
        }
        double best = 1e300;
        for (int rep = 0; rep < 3; ++rep) {
            cudaError_t ee = cudaEventRecord(t0, st);
            if (ee != cudaSuccess) return cuda_fail(ee);
            int r = batched_body(b, X, x_dtype, factors, n_factors, (char *)ws, st, U_out, V_out);
            if (r != USTAT_OK) return r;
            ee = cudaEventRecord(t1, st);
            if (ee == cudaSuccess) ee = cudaEventSynchronize(t1);
            if (ee != cudaSuccess) return cuda_fail(ee);
            float f = 0.f;
            cudaEventElapsedTime(&f, t0, t1);
            if (rep > 0) best = std::min(best, (double)f);
        }
        *ms = best;
        return USTAT_OK;
    };
    double best_ms = 1e300;
    int best_lanes = b->lanes;
    // lane count first (default GEMM variants), then the GEMM variant of each
    // size class present in the batch, one class at a time
    for (int L = 1; L <= std::min(b->max_lanes, (int)b->n.size()); L *= 2) {
        b->lanes = L;
        batched_schedule(b);
        double ms = 0.0;
        rc = timed(&ms);
        if (rc != USTAT_OK) break;
        if (ms < best_ms) {
            best_ms = ms;
            best_lanes = L;
        }
    }
    b->lanes = best_lanes;
    batched_schedule(b);
    if (rc == USTAT_OK && is_tc_mode(P.precision)) {
        bool present[4] = {false, false, false, false};
        for (int64_t v : b->n) present[tc_size_class(v)] = true;
        // raster groups x tile shapes (bf16x3: 3 shapes; bf16x4: 2; tf32: 1)
        std::vector<int> vars;
        bool rbf_build = false;
        for (auto &op : P.ops)
            rbf_build |= op.kind == OP_KBUILD && P.factor_kind[op.factor] == USTAT_RBF && !wide_storage(P.precision);
        // RBF builds: the tensor-core Gram build (bits 4-5 clear), or the CUDA-core
        // build with either tile (bit 5 set, bit 4 the tile)
        const int builds[3] = {0, 32, 48};
        for (int kb = 0; kb < (rbf_build ? 3 : 1); ++kb)
            for (int shape = 0; shape < 3; ++shape) {
                if (P.precision == USTAT_BF16X4 && shape == 1) continue;
                if (P.precision == USTAT_BF16X5 && shape != 2) continue;
                if (P.precision == USTAT_TF32 && shape > 0) continue;
                for (int gr = 0; gr < 4; ++gr) vars.push_back(gr | (shape << 2) | builds[kb]);
            }
        for (int c = 0; c < 4 && rc == USTAT_OK; ++c) {
            if (!present[c]) continue;
            int best_v = P.tc_variant[c];
            for (int v : vars) {
                if (v == best_v) continue;
                const int keep = P.tc_variant[c];
                P.tc_variant[c] = v;
                double ms = 0.0;
                rc = timed(&ms);
                if (rc != USTAT_OK) break;
                if (ms < best_ms * 0.995) {
                    best_ms = ms;
                    best_v = v;
                }
                P.tc_variant[c] = keep;
            }
            P.tc_variant[c] = best_v;
        }
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (rc != USTAT_OK) return rc;
    if (lanes_out) *lanes_out = b->lanes;
    if (ms_out) *ms_out = best_ms;
    return USTAT_OK;
}

}  // extern "C"
