// Host-side launchers of the engine's CUDA kernels (internal).
#pragma once

#include <cstdint>
#include <vector>
#include <cuda_runtime.h>

namespace ustat {

// ---- tensorization and vector ops (k_elem.cu)
// The kernels that read the caller's inputs (X, MATRIX and VECTOR data) set bit
// kErrWordNonfinite of the device error word *err (may be null) when an input
// value is NaN or infinite.
constexpr int kErrWordTimeout = 1, kErrWordNonfinite = 2;
// Xw = working copy of X: float64 when fp64, else float32 (row-major n x d).
cudaError_t launch_xconvert(const void *X, int x_dtype, int64_t n, int d, void *Xw, bool fp64, int *err,
                            cudaStream_t s);
// K(i,j) = exp(-||x_i - x_j||^2 / param) (kind RBF) or (x_i . x_j) / param (LINEAR).
cudaError_t launch_kbuild(int kind, double param, const void *Xw, bool fp64, int64_t n, int d,
                          int zero_diag, void *K, cudaStream_t s);
// RBF kernel matrix (float32) fused with its split into `planes` bf16 slices of
// row scale 1 (slices may be null: K only) and with up to 4 reductions of its
// entrywise powers: red_vec[q] ? red_out[q][i] += sum_j K_ij^red_pow[q]
//                              : *red_out[q] += sum_ij K_ij^red_pow[q].
// X is read as float32 (Xw) or as float64 (Xd, rounded to float32 while staged).
cudaError_t launch_kbuild_rbf(const float *Xw, const double *Xd, int64_t n, int d, double param, int zero_diag,
                              float *K, void *slices, int64_t ldp, int lead_bits, int planes, float *scales, int nred,
                              const int *red_pow, const int *red_vec, double *const *red_out, int upper_only,
                              int tile64, int *err, cudaStream_t s);
// The same RBF build with the squared distances from the Gram matrix X X^T on the
// tensor cores (k_gram_tc.cu): X (float64 or float32, d <= 256) is read
// directly; `scratch` (256-byte aligned, kbuild_rbf_tc_scratch_bytes) holds X's
// digit planes, row scales and squared norms.
size_t kbuild_rbf_tc_scratch_bytes(int64_t n, int d);
cudaError_t launch_kbuild_rbf_tc(const void *X, int x_dtype, int64_t n, int d, double param, int zero_diag, float *K,
                                 void *slices, int64_t ldp, int lead_bits, int planes, float *scales, int nred,
                                 const int *red_pow, const int *red_vec, double *const *red_out, int upper_only,
                                 void *scratch, int *err, cudaStream_t s);
// The same build in two parts, for the memory-lean evaluation: the prep (X's
// digit planes, scales and norms into `scratch`, once per evaluation), then any
// number of windows: the entries of rows row0 .. row0 + rows - 1 and columns
// col0 .. col0 + cols - 1 (row0, col0 multiples of 128), each computed once (no
// mirror).  K (may be null) and scales keep global indices (K[j * n + k],
// scales[j]; the caller offsets pointers of buffers that hold only the window);
// the digit planes hold row j at j - srow0 with plane stride splane elements;
// reductions add every window entry once (vector reductions: row sums).
cudaError_t launch_gram_rbf_prep(const void *X, int x_dtype, int64_t n, int d, void *scratch, int *err,
                                 cudaStream_t s);
cudaError_t launch_gram_rbf_window(int64_t n, int d, double param, int zero_diag, float *K, void *slices,
                                   int64_t ldp, int lead_bits, int planes, float *scales, int nred,
                                   const int *red_pow, const int *red_vec, double *const *red_out, int64_t row0,
                                   int64_t rows, int64_t col0, int64_t cols, int64_t srow0, int64_t splane,
                                   void *scratch, int *err, cudaStream_t s);
// Linear kernel of a float32 X into a float64 K (float64-storage modes): the
// double-float dot product, unrounded.
cudaError_t launch_kbuild_linear_wide(const float *X, int64_t n, int d, double param, int zero_diag, double *K,
                                      cudaStream_t s);
cudaError_t launch_loadmat(const double *src, int64_t n, bool fp64, int zero_diag, int complement, void *dst,
                           int *err, cudaStream_t s);
// LOWRANK (data = [P | Q], n x 2r: F = P Q') or DIST (data = Y, n x r: F(i, j) =
// ||y_i - y_j||) factor matrices in float64 arithmetic, stored in the mode's type.
cudaError_t launch_pairs(int kind, const double *data, int r, int64_t n, bool fp64, int zero_diag, void *dst,
                         int *err, cudaStream_t s);
cudaError_t launch_unary_tanh(const void *X, int x_dtype, int64_t n, int d, const double *w,
                              double *out, int *err, cudaStream_t s);
cudaError_t launch_copyvec(const double *src, int64_t n, double *dst, int *err, cudaStream_t s);
cudaError_t launch_diag(const void *M, bool fp64, int64_t n, double *out, cudaStream_t s);
cudaError_t launch_vmul(const double *a, const double *b, int64_t n, double *out, cudaStream_t s);
// out(i) = F(x_i, x_i) of factor kind `kind` from its own data in float64 (X for
// LINEAR / RBF, the caller's matrix Mc for MATRIX); 0 when zero_diag.
cudaError_t launch_factor_diag(int kind, double param, const void *X, int x_dtype, int d, const double *Mc,
                               int64_t n, int zero_diag, double *out, cudaStream_t s);
cudaError_t launch_vsum(const double *u, int64_t n, double *out, cudaStream_t s);
// *out += sum_i u(i) a(i)
cudaError_t launch_vdot(const double *u, const double *a, int64_t n, double *out, cudaStream_t s);

// ---- tiled elementwise / reduction ops over up to 4 oriented matrix terms (k_hb.cu)
enum TileMode : int { TILE_HADAMARD = 0, TILE_FREDUCE = 1, TILE_GEMV = 2 };
struct TileTerms {
    const void *M[4];
    int trans[4];
    int nt;
};
// HADAMARD: out(i,j) = prod_t term_t(i,j)                       (out: matrix)
// FREDUCE : *out += sum_ij prod_t term_t(i,j) a(i) b(j)          (out: double scalar)
// GEMV    : out(j) += sum_i a(i) prod_t term_t(i,j)              (out: double vector)
cudaError_t launch_tile_op(int mode, const TileTerms &tt, bool fp64, int64_t n, const double *a,
                           const double *b, void *out, cudaStream_t s);

// ---- several reductions / GEMVs over the same matrices in one pass (k_hb.cu)
// Every term is read untransposed (value(i, j) = M[i][j]).
//   FREDUCE: *out += sum_ij prod_t M_t(i,j) a(i) b(j)
//   GEMV   : out(j) += sum_i a(i) prod_t M_t(i,j)
constexpr int kMhbMats = 4, kMhbOps = 6, kMhbGemv = 2;
struct MhbOp {
    int kind;             // TILE_FREDUCE or TILE_GEMV
    int nt;
    int mat[4];           // indices into MhbArgs::M
    int ex[4];            // filled by launch_mhb: multiplicity of each matrix
    const double *a, *b;
    double *out;
};
struct MhbArgs {
    int64_t n;
    int nmat;
    const void *M[kMhbMats];
    int nops;
    MhbOp op[kMhbOps];
};
cudaError_t launch_mhb(const MhbArgs &g, bool fp64, cudaStream_t s);

// ---- SIMT GEMMs in float32 / float64 (k_gemm_simt.cu)
// One fused reduction: *out += sum_jk C(j,k)^pow W(j,k) a(j) b(k)
struct SimtRed {
    const void *W;
    int transW;
    const double *a, *b;
    int pow;
    double *out;
};
struct SimtGemmArgs {
    int64_t n;
    const void *A;  int transA;     // A(i, j)
    const void *B;  int transB;     // B(i, k)
    const double *u;                // along i, may be null
    // epilogue
    void *C;                        // stored product C(j, k), row-major n x n (may be null)
    int nred;                       // fused reductions (0..4)
    SimtRed red[4];
    int symmetric;                  // C = C^T, reductions symmetric: upper tiles only
    // GEMM3 (batched over index bb; one reduction red[0]): u'(i) = u(i) Ab(i, bb),
    // extra weights Wbc(bb, j), Wbd(bb, k), ub(bb)
    const void *Ab; int transAb;
    const void *Wbc; int transWbc;
    const void *Wbd; int transWbd;
    const double *ub;
    int gemm3;
};
cudaError_t launch_gemm_simt(const SimtGemmArgs &g, bool fp64, cudaStream_t s);

// ---- Moebius combination (k_elem.cu)
constexpr int kCombineMaxParts = 877;
constexpr int kCombineMaxScal = 6;
struct CombineEntry {
    int mu;
    unsigned short sid[kCombineMaxScal];   // scalar slot index, 0xffff = none
    unsigned char nfree;
    unsigned char evaluated;
};
// V_pi = prod_q scal[sid] * n^nfree (0 if not evaluated); U = sum mu V.
// A non-zero *err (a bounded device wait gave up) turns U and V into NaN.
cudaError_t launch_combine(const CombineEntry *entries, int nparts, int m, const double *scal, const int *err,
                           int64_t n, double *U_out, double *V_out, cudaStream_t s);

// ---- tensor-core path (k_gemm_tc.cu)
// digits of the leading bf16 slice for a contraction of length K (exact integer
// accumulation of the leading product needs K * 4^w1 <= 2^24)
int split_lead_bits(int64_t K);
// Operand X(j, i) = M(i, j) u(i) (trans = 0: column j of M; trans = 1: row j),
// written K-major:
//   split bf16: `planes` slices [planes][n][ldp] plus float row scales [n]  (launch_split)
//   float32 tf32-rounded copy [n][ldp]                                        (launch_prep)
// With diag_out, a row whose diagonal entry X(j, j) dominates (more than four
// times its largest other entry; every row for a column source) leaves it out of
// the digits and of the row scale and writes it to diag_out[j] (float64; 0 for a
// row that keeps it): the GEMM adds the left-out terms exactly (TcGemmArgs::dA,
// dB).
cudaError_t launch_split(const void *M, bool wide, int trans, const double *u, int64_t n, int64_t ldp,
                         int lead_bits, int planes, void *slices, float *scales, double *diag_out, cudaStream_t s);
cudaError_t launch_prep(const float *M, int trans, const double *u, int64_t n, int64_t ldp,
                        float *out, cudaStream_t s);
// One fused reduction of the product C: *out += sum_jk C(j,k)^pow W(j,k) a(j) b(k)
// (W, a, b may be null = all ones; W read with orientation transW).
struct TcRed {
    const void *W;                           // float, or double with `wide`
    int transW;
    const double *a, *b;
    int pow;
    double *out;
};
struct TcGemmArgs {
    int64_t n, ldp;
    const void *opA; const float *scaleA;   // K-major operand of A (slices or prep)
    const void *opB; const float *scaleB;
    int lead_bits;
    void *C;                                 // stored product (may be null): float, double with `wide`
    int nred;                                // fused reductions (0..4)
    TcRed red[4];
    int symmetric;                           // C = C^T and every reduction symmetric
    int *err;                                // device error word (bounded waits)
    int group_rows;                          // tile rows per raster group (0: 8)
    // GEMM3 batch (s = 3 step on the tensor cores): `batch` > 0 products, one per
    // bb = bb0 .. bb0 + batch - 1, whose A operands are consecutive in opA
    // ([batch][planes][n][ldp], scales [batch][n]); one reduction red[0] with the
    // extra weights Wbc(bb, j) on rows, Wbd(bb, k) on columns and ub(bb)
    int batch, bb0;
    int split_tail;                          // set by the launcher: trailing tiles split in halves
    const void *Wbc; int transWbc;
    const void *Wbd; int transWbd;
    const double *ub;
    // float64 storage (bf16x4 only): W, Wbc, Wbd and C are double, and the epilogue
    // forms the entries and the reductions in float64
    int wide;
    // with `wide` and `batch` (the s = 3 step): the epilogue runs in float32 with
    // float32 copies of W, Wbc and Wbd (the four accumulators summed in float32)
    int wide_f32;
    // Diagonal correction (non-batched products).  An operand split with its
    // diagonal left out (X(j, j) = 0 in the digits, its value in dA / dB, float64)
    // misses the terms i = j of C(j, k) = sum_i XA(j, i) XB(k, i); the epilogue adds
    //   dA[j] XB(k, j) + XA(j, k) dB[k] - [j = k] dA[j] dB[j]
    // from the operands' sources: XA(j, k) = MA(k, j) uA(k), XB(k, j) = MB(j, k) uB(j),
    // read as MA[j][k] when rowA (else MA[k][j]) and MB[j][k] when rowB (else
    // MB[k][j]); dA or dB null: that operand keeps its diagonal.
    const double *dA, *dB;
    const void *MA, *MB;                     // float, or double with `wide`
    int rowA, rowB;
    const double *uA, *uB;
    // row shard: the product's tiles are divided into shard_count contiguous
    // ranges of its walk and only range shard_rank is computed (shard_count > 1;
    // reductions only: the ranks' scalars sum to the product's); the launcher sets
    // tile_lo / tile_hi
    int shard_rank, shard_count;
    int tile_lo, tile_hi;
    // set by the launcher from set_tc_debug: the limit of every mbarrier wait in SM
    // cycles (0: the default, about two seconds) and the stalled-producer test hook
    long long wait_limit;
    int debug_stall;
    // window (memory-lean evaluation; rows = 0: the whole product): only rows
    // row0 .. row0 + rows - 1 and columns col0 .. col0 + cols - 1 of the product,
    // reductions only.  opA holds the digit planes of just those rows of A
    // ([planes][rows][ldp]) and opB of those rows of B ([planes][cols][ldp]); every
    // other array keeps global indices (scaleA[j], scaleB[k], W[j * n + k], the
    // reduction vectors), so the caller offsets the pointers of arrays that hold
    // only the window.  Symmetric needs row0 = col0 and rows = cols.  Every tile's
    // reductions are multiplied by wscale (0: 1).
    int64_t row0, col0, rows, cols;
    double wscale;
    // grouped launch (set by launch_gemm_group): gcount products, their arguments
    // and tensor maps (A, B per product) in device memory, tile prefix sums gstart
    const TcGemmArgs *gargs;
    const void *gmaps;
    const int *gstart;
    int gcount;
};
// Test hook of the bounded waits (off by default): every later tensor-core GEMM
// launch of this process uses `wait_limit` cycles (0 = default) as its wait limit
// and, with `stall`, issues no TMA copy, so its first wait runs out.
void set_tc_debug(long long wait_limit, int stall);
// The wait limit set by set_tc_debug (0: the default).
long long tc_debug_wait_limit();
// shape: 0 = 128 x 128 tiles, 128-byte k-blocks, two stages; 1 = 128 x 64 tiles,
// three stages (no symmetric tile skipping); 2 = 128 x 128 tiles, 64-byte
// k-blocks, four stages (bf16x4: 0 = 128 x 64 tiles, two stages; 2 = 128 x 128
// tiles, 64-byte k-blocks, three stages)
cudaError_t launch_gemm_bf16x3(const TcGemmArgs &g, int shape, cudaStream_t s);
// One persistent bf16x3 launch over the tiles of `count` products (a group): the
// host builds the group's device image (each entry's A and B tensor maps, its
// arguments, the tile prefix sums) with gemm_group_image for the device address
// it will be copied to (gemm_group_bytes bytes, 256-byte aligned) and returns the
// total tile count (-1: an entry the grouped form does not take: batched, window,
// shard or float64-storage products); launch_gemm_group then runs all tiles, each
// entry's reductions added to its own outputs.  Entries keep their own error
// words; a bounded wait that gives up sets every entry's.
size_t gemm_group_bytes(int count);
int gemm_group_image(const TcGemmArgs *items, int count, int shape, const void *dev_base, std::vector<char> &host);
cudaError_t launch_gemm_group(const void *dev_base, int count, int total_tiles, int shape, int *err, cudaStream_t s);
cudaError_t launch_gemm_bf16x4(const TcGemmArgs &g, int shape, cudaStream_t s);
// five slices, 128 x 128 tiles, 64-byte k-blocks; float64 storage only
cudaError_t launch_gemm_bf16x5(const TcGemmArgs &g, cudaStream_t s);
// Digit planes of the s = 3 step's A operands for bb = bb0 .. bb0 + nb - 1:
// X_bb(j, i) = A(i, j) u(i) Ab(i, bb) with A(i, j) = trans ? M[j][i] : M[i][j] and
// Ab(i, bb) = transAb ? Mb[bb][i] : Mb[i][bb]; slices [nb][planes][n][ldp],
// scales [nb][n].
cudaError_t launch_split_g3(const void *M, bool wide, int trans, const double *u, const void *Mb, int transAb,
                            int64_t bb0, int nb, int64_t n, int64_t ldp, int lead_bits, int planes, void *slices,
                            float *scales, cudaStream_t s);
cudaError_t launch_gemm_tf32(const TcGemmArgs &g, cudaStream_t s);
// float64 -> float pair (hi, lo; lo may be null: float64 -> float), `total` entries.
cudaError_t launch_f64_pair(const double *M, int64_t total, float *hi, float *lo, cudaStream_t s);
// The s = 3 step's A operands of the float64-storage modes, from float-pair copies
// (Mh, Ml) of a row-major source read along rows (A(i, j) = M[j][i]), in float32
// double-float arithmetic; n <= kPairSplitMaxN.  Layout as launch_split_g3.
constexpr int64_t kPairSplitMaxN = 24576;
cudaError_t launch_split_g3_pair(const float *Mh, const float *Ml, const double *u, const double *Mb, int transAb,
                                 int64_t bb0, int nb, int64_t n, int64_t ldp, int lead_bits, int planes, void *slices,
                                 float *scales, cudaStream_t s);

}  // namespace ustat
