// Internal declarations of libmlblup: context layout, cell tables and the
// kernel launchers shared between translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/mlblup.h"
#include "matern.cuh"

namespace mlb {

constexpr int kMaxDim = 16;       // largest point dimension d
constexpr int kTile = 64;         // largest local basis size on the assembled path

// Numbers of one cell of the kd-tree, level-order id g = 2^l - 1 + k.
// s = size of the local basis (points for a leaf, children's scaling vectors
// otherwise), a = scaling vectors, k = s - a wavelets.
struct CellTables {
    int* beg = nullptr;     // first kd position of the cell's points
    int* end = nullptr;
    int* s = nullptr;
    int* a = nullptr;
    int* k = nullptr;
    int64_t* vOff = nullptr;   // offset of the s x s factor V in the V pool
    int64_t* rOff = nullptr;   // offset of the a x p moment factor R in the R pool
    int64_t* wOff = nullptr;   // first row of the cell's wavelets in W (finest level first)
    int64_t* sOff = nullptr;   // first scaling index of the cell within its level
    int64_t* wLoc = nullptr;   // first wavelet index of the cell within its level
    double* lo = nullptr;      // bounding box of the cell's points (ncell x d)
    double* hi = nullptr;
    double* diam = nullptr;    // Euclidean diagonal of that box
};

struct HostCell {
    int beg, end, s, a, k;
    int64_t vOff, rOff, wOff, sOff, wLoc;
};

// Panels of the assembled C~_W: every row cell c owns a dense k_c x ncols_c
// row-major panel holding all its blocks side by side (columns in global
// wavelet order) and one column-index list shared by its k_c rows.
struct Panels {
    int64_t nnz = 0, blocks = 0, colTotal = 0, nnzUnique = 0, stored = 0;
    // ncols holds the padded panel width (multiple of 4); nnz counts real entries
    int* ncols = nullptr;       // per cell
    int64_t* valOff = nullptr;  // per cell, into vals
    int64_t* colOff = nullptr;  // per cell, into colidx
    int* colidx = nullptr;
    int* bcol = nullptr;        // ncell x ncell: column offset of block (c, e) in panel c, or -1
    int* rowCell = nullptr;     // per wavelet row: its cell
    double* vals = nullptr;     // FP64 values
    float* vals32 = nullptr;    // FP32 copy (mixed precision)
    // FP32 product: one CTA per (cell, first row, first column, segment) of at
    // most kItemRows rows and kSegCols columns, heaviest first; the segments'
    // partial rows go to ypart (segment-major) and are summed in order
    int4* work = nullptr;
    int nwork = 0;
    int* nseg = nullptr;        // per cell: column segments of its panel
    double* ypart = nullptr;    // nsegMax x nwav partial products
    int nsegMax = 0;
};

// Rows and columns of one work item of the FP32 product (one CTA of 8 warps,
// up to 4 rows per warp; the column range a multiple of the 256-column chunk).
constexpr int kItemRows = 32;
constexpr int kSegCols = 8192;

// Upper bound on the FP32 product's work items: the cells hold nwav <= N rows
// and at most N columns, so the count is at most
// (ncell + N / kItemRows) x ceil(N / kSegCols).
// The symmetric product's items (sym_plan, at least 512 columns each) number
// at most ceil(N / 128) x (ceil(N / 512) + 1); the bound covers both.
inline size_t max_work_items(int ncell, int64_t N) {
    const size_t panels = ((size_t)ncell + (size_t)(N / kItemRows) + 1) * (size_t)((N + kSegCols - 1) / kSegCols);
    const size_t sym = (size_t)((N + 127) / 128) * (size_t)((N + 511) / 512 + 1);
    return panels > sym ? panels : sym;
}

// Symmetric packed storage of a complete C~_W in FP32 (mixed path, every
// cell pair admissible): each symmetric pair of entries is stored once.  The
// wavelet rows are grouped in blocks of kSymRows; block b keeps its rows from
// its own first column (b kSymRows) to the last, i.e. its diagonal square in
// full and everything to the right of it, over sym_width(nwav, b) columns (a
// multiple of kSymTile, zero padded).  Those columns are cut into tiles of
// kSymTile columns, each stored contiguously (the block's rows one after the
// other, kSymTile values each), so one tile is one contiguous copy.  The
// product streams every stored value once and applies it twice (B x to the
// block's rows and B^T x to the columns' rows).  Work items are (block,
// segment of `seg` columns, a multiple of 256 chosen by the autotuner),
// heaviest first; an item's row sums go to
// rowpart (by segment) and its column sums to colpart (by block), both summed
// in a fixed order by the consumer, so the product is deterministic.
constexpr int kSymRows = 128;
constexpr int kSymTile = 64;

__host__ __device__ inline int64_t sym_width(int64_t nwav, int b) {
    return ((nwav - (int64_t)b * kSymRows) + kSymTile - 1) / kSymTile * kSymTile;
}
__host__ __device__ inline int sym_nseg(int64_t nwav, int b, int seg) {
    return (int)((sym_width(nwav, b) + seg - 1) / seg);
}

struct SymPanels {
    int nblk = 0;               // row blocks
    int64_t stored = 0;         // FP32 values stored
    float* vals = nullptr;
    int64_t* off = nullptr;     // per block: offset of its first value
    int2* work = nullptr;       // (block, segment), heaviest first
    int nwork = 0;
    int nworkCap = 0;
    int seg = 0;                // columns per work item
    int nsegMax = 0;
    int nsegCap = 0;            // segments the row-partial buffer holds per right-hand side
    int nrhs = 0;               // right-hand sides the partial buffers hold
    float* rowpart = nullptr;   // nrhs x nsegCap x nwav (FP32 sums)
    float* colpart = nullptr;   // nrhs x nblk x nwav
    float* xh = nullptr;        // nrhs x xld: FP32 high parts of the vectors multiplied
    float* xl = nullptr;        //             and their low parts (x = h + l to about 2^-48)
    int64_t xld = 0;            // nwav rounded up past the widest padded row, zero beyond nwav
    int* err = nullptr;         // device flag: bit 0 set when a bounded wait of the product gave up
};

// Data box centre and per-axis scale sqrt(theta_k) of the kernel distance
// (1 on every axis for the isotropic distance); the kernels read coordinates
// as (x - c) sc or x sc.
struct KGeo {
    double c[kMaxDim];
    double sc[kMaxDim];
};

struct PcgState {
    double rz, rr, bb, alpha, beta, pq;
    int it, done, status;
    unsigned ticket;     // CTAs of the current launch that have finished (last-CTA reductions)
};

// Device allocations of one lifetime.  release() frees them all; callers
// synchronise every stream that uses them first (cudaFree need not wait).
struct Arena {
    std::vector<void*> ptrs;
    void release();
};

}  // namespace mlb

struct mlb_ctx {
    mlb_opts opts;
    cudaStream_t own_stream = nullptr;
    cudaStream_t stream = nullptr;
    std::string err;
    int state = 0;                 // 0 empty, 1 basis, 2 assembled, 3 solved
    int64_t launches = 0;          // kernels launched by this context
    int ksum_variant = 1;          // launch shape of the FP32 kernel sum (autotuned)
    int nsm = 0;                   // SMs of the context's device
    double* ksum_part = nullptr;   // kernel sums: partial sums of the source chunks
    int64_t ksum_part_cap = 0;     // its length in doubles

    // basis
    int64_t N = 0, nwav = 0;
    int d = 0, p = 0, w = 0, t = 0, ncell = 0;
    std::vector<mlb::HostCell> hcells;
    std::vector<int64_t> sumA, sumK, levelBase, sbase;   // per level
    std::vector<int> hperm;
    double box_lo[mlb::kMaxDim], box_hi[mlb::kMaxDim];
    double* xs = nullptr;          // N x d points in kd order
    float* xs32 = nullptr;         // mixed: FP32 offsets of the points from the data box centre
    float* xs32lo = nullptr;       // mixed: low parts of those offsets (double-float coordinates)
    float* xl32 = nullptr;         // mixed: FP32 offsets of the points from their leaf's box centre
    float* xl32lo = nullptr;       // mixed: low parts of the leaf offsets
    double* leafctr = nullptr;     // mixed: box centre of every cell (ncell x d)
    int* perm = nullptr;           // kd position -> caller index
    int* alpha = nullptr;          // p x d monomial exponents
    double* X = nullptr;           // N x p design matrix, kd order
    double* XtXf = nullptr;        // p x p Cholesky factor of X^T X
    double* V = nullptr;           // pool of the cells' s x s orthogonal factors
    double* R = nullptr;           // pool of the cells' a x p moment factors
    double* sbuf = nullptr;        // scaling coefficients of every level (transforms)
    int* flag = nullptr;           // device error flags
    mlb::CellTables cells;
    mlb::Arena arena_basis;

    // assembly
    mlb_theta theta{};
    mlb::KernelFn kfn{};           // covariance function of the assembly (kernelfn.cu)
    mlb::KGeo kgeo{};              // data box centre and per-axis distance scales
    const float* kxs32 = nullptr;  // FP32 coordinates the kernels read: the basis arrays,
    const float* kxs32lo = nullptr;//   or scaled copies for an anisotropic distance
    const float* kxl32 = nullptr;
    const float* kxl32lo = nullptr;
    const double* kctr = nullptr;
    double tau_factor = 0;
    mlb::Panels pan;
    mlb::SymPanels sym;            // mixed path, complete pattern: each symmetric pair stored once
    bool allow_sym = true;         // false: keep the FP32 row panels instead (batched small systems)
    int sym_variant = 0;           // form of the symmetric product (autotuned): 0 loads, 1 bulk-copy pipeline
    double* diag = nullptr;        // diag(C~_W)
    double ms_assemble = 0;
    mlb::Arena arena_asm;

    // solve
    double* gW = nullptr;          // gamma_W
    double* gamma = nullptr;       // gamma-hat, kd order
    double* beta = nullptr;        // beta-hat
    double* vec = nullptr;         // PCG work vectors
    double* partial = nullptr;
    mlb::PcgState* pcg = nullptr;
    mlb::Arena arena_solve;
    mlb_info last_info{};
};

namespace mlb {

// ---- error helpers -------------------------------------------------------
mlb_status fail(mlb_ctx* ctx, mlb_status s, const std::string& msg);
mlb_status cuda_fail(mlb_ctx* ctx, cudaError_t e, const char* where);
void* dalloc(mlb_ctx* ctx, Arena& a, size_t bytes);
// Frees one allocation of the arena after the context's stream has drained:
// cudaFree is documented only as possibly synchronising, and kernels queued
// on the stream may still write the buffer.  Freed memory goes straight back
// to the device allocator, where another host thread's cudaMalloc can take it
// for work on another stream.
void dfree(mlb_ctx* ctx, Arena& a, void* p);
// largest dynamic shared memory a block may opt in to on the current device
int max_smem_optin();
// opts a kernel in to all the dynamic shared memory its static share leaves free;
// one constant per kernel, so contexts on different host threads cannot race
mlb_status allow_max_dynamic_smem(mlb_ctx* ctx, const void* func, const char* name);

#define MLB_CUDA(ctx, call)                                        \
    do {                                                           \
        cudaError_t e__ = (call);                                  \
        if (e__ != cudaSuccess) return mlb::cuda_fail(ctx, e__, #call); \
    } while (0)

#define MLB_CHECK_LAUNCH(ctx, what)                                   \
    do {                                                              \
        (ctx)->launches += 1;                                         \
        cudaError_t e__ = cudaGetLastError();                         \
        if (e__ != cudaSuccess) return mlb::cuda_fail(ctx, e__, what); \
    } while (0)

// ---- launchers (defined in the .cu files) ---------------------------------
// basis.cu
mlb_status build_design(mlb_ctx* ctx);
mlb_status build_factors(mlb_ctx* ctx);
mlb_status apply_W_dev(mlb_ctx* ctx, const double* v_kd, double* out);    // N (kd) -> nwav
mlb_status apply_Wt_dev(mlb_ctx* ctx, const double* u, double* out_kd);   // nwav -> N (kd)
mlb_status gather_kd(mlb_ctx* ctx, const double* v_user, double* v_kd);   // caller -> kd order
mlb_status scatter_kd(mlb_ctx* ctx, const double* v_kd, double* v_user);  // kd -> caller order
// kernelfn.cu: kind, scale and table of the covariance function, scaled
// coordinates of an anisotropic distance (allocations in arena_asm)
mlb_status setup_kernel_fn(mlb_ctx* ctx);
// assemble.cu
mlb_status assemble_dev(mlb_ctx* ctx);
// symv.cu: the symmetric packed FP32 storage (from the FP64 panels of a
// complete pattern) and its product
mlb_status build_sym(mlb_ctx* ctx);
// partial buffers for nrhs simultaneous products (grown on demand)
mlb_status sym_reserve(mlb_ctx* ctx, int nrhs);
// products of the nrhs vectors x (nrhs x nwav) into the partial buffers; part
// (nrhs x nwork) and st (nrhs states) may be nullptr outside the PCG.
// presplit: the FP32 parts of x are already in ctx->sym.xh / xl (the PCG's
// vector updates write them)
void sym_launch(mlb_ctx* ctx, const double* x, int nrhs, double* part, PcgState* st, bool presplit = false);
// out = the sums of the partials of right-hand side 0
void sym_reduce(mlb_ctx* ctx, double* out);
// solve.cu
mlb_status cw_matvec_dev(mlb_ctx* ctx, const double* u, double* out);
mlb_status solve_dev(mlb_ctx* ctx, const double* Z_kd, mlb_info* info);
mlb_status trend_dev(mlb_ctx* ctx, const double* Z_kd);
// ksum.cu
mlb_status kernel_sum_dev(mlb_ctx* ctx, const double* targets, int64_t M, const double* a_kd,
                          double* out, bool add_trend);
// out_k = sum_j f(|y_k - s_j|) w_j over Ns sources s (nullptr: the data points,
// kd order); f = phi or d phi / d log(rho); optional trend k(y)^T beta.
// On the mixed path `accurate` selects double-float kernel values (one-shot
// sums: trend step, prediction, gradient) instead of FP32 ones (the kernel sum
// inside every matrix-free PCG iteration).
mlb_status kernel_sum_general(mlb_ctx* ctx, const double* targets, int64_t M, const double* sources,
                              int64_t Ns, const double* weights, double* out, bool add_trend, bool deriv,
                              bool accurate = true);
// picks the FP32 kernel-sum launch shape for this context (ksum.cu)
mlb_status tune_kernel_sum(mlb_ctx* ctx);
// ksum_tc.cu: the matrix-free product's kernel sum (targets = sources = the
// data points) on the tensor cores; false when the dimension or covariance
// kind has no tensor-core form (then nothing is launched)
constexpr int kKsumFormTC = 6;   // ksum_variant value of the tensor-core form
bool ksum_tc_supported(const mlb_ctx* ctx);
bool ksum_tc_self(mlb_ctx* ctx, const double* a, double* out);
// solve.cu: PCG on C~_W x = b (nwav vectors on the device)
mlb_status pcg_run(mlb_ctx* ctx, const double* b, double* x, mlb_info* info);
// kRhs simultaneous PCG solves on the FP32 panels (one pass over C~_W per iteration)
constexpr int kRhs = 4;
size_t pcg_multi_work_doubles(const mlb_ctx* ctx);
mlb_status pcg_run_multi(mlb_ctx* ctx, const double* b, double* x, double* work, int* iters);
// grad.cu
mlb_status grad_dev(mlb_ctx* ctx, const double* targets, int64_t M, const double* y, double* out3);
mlb_status mse_dev(mlb_ctx* ctx, const double* targets, int64_t M, double* out);

}  // namespace mlb
