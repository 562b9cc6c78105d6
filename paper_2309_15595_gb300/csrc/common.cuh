// Internal declarations shared by the kernel translation units and the host
// driver. Complex128 values are double2 (x = real, y = imaginary), matrices are
// column-major with explicit leading dimensions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/chase.h"

namespace chase {

// ----------------------------------------------------------- complex helpers
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ double2 cmulc(double2 a, double2 b) {  // conj(a) * b
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__host__ __device__ __forceinline__ double2 cadd(double2 a, double2 b) {
  return make_double2(a.x + b.x, a.y + b.y);
}
__host__ __device__ __forceinline__ double2 csub(double2 a, double2 b) {
  return make_double2(a.x - b.x, a.y - b.y);
}
__host__ __device__ __forceinline__ double2 cscale(double s, double2 a) {
  return make_double2(s * a.x, s * a.y);
}
__host__ __device__ __forceinline__ double2 conjz(double2 a) { return make_double2(a.x, -a.y); }
__host__ __device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }
// acc += a * b with four fused multiply-adds
__device__ __forceinline__ void cfma(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}

__host__ __device__ inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Runs f() once per CUDA device (the one current when called), thread-safe:
// kernel attributes such as the dynamic shared-memory limit are per device, and
// solves run from several host threads at once.
constexpr int kMaxDevices = 64;
template <typename F>
void once_per_device(std::once_flag (&flags)[kMaxDevices], F&& f) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    f();
    return;
  }
  std::call_once(flags[dev], f);
}
// Reports a failed CUDA call (with the pending CUDA error, if any) on stderr and
// returns CHASE_ERR_CUDA; used by every CUDA-error return of the library.
int report_cuda_failure(const char* file, int line);
#define CHASE_CUDA_FAIL() ::chase::report_cuda_failure(__FILE__, __LINE__)
// Number of SMs of the current device (cached per device).
int num_sms();

// Process-wide count of kernel launches issued by this library.
void count_launch();
long long launch_count();

// ------------------------------------------------------------- GEMM (FP64)
// Epilogue of the complex FP64 GEMM  P = A * B  (M x n, K inner).
enum EpiMode { EPI_STORE = 0, EPI_FILTER = 1, EPI_RESID = 2 };
struct Epilogue {
  int mode;
  double alpha, beta, gamma;  // filter: out = alpha (P - gamma X) + beta Y
  const double2* X;           // filter/resid: the B operand read element-wise
  int64_t ldx;
  double2* Y;                 // store / filter destination
  int64_t ldy;
  const double* theta;        // resid: Ritz values per column
  double* partial;            // resid: [row_tile + col * n_row_tiles] sums of |.|^2
};

// P = A (M x K) * B (K x n); A column-major (lda), B column-major (ldb).
cudaError_t zgemm_nn(cudaStream_t s, int64_t M, int64_t n, int64_t K, const double2* A,
                     int64_t lda, const double2* B, int64_t ldb, const Epilogue& ep);
// Number of 64-row tiles the residual epilogue writes partials for.
int64_t zgemm_row_tiles(int64_t M);
// Fixed-order reduction of the residual partials: out[j] = sqrt(sum_t partial).
cudaError_t resid_reduce(cudaStream_t s, const double* partial, int64_t ntiles, int64_t n,
                         double* out);

// Gram products G = X^H Y (m x n) over K rows, split-K with a deterministic
// reduction. hermitian: X == Y, only upper tiles computed, G made exactly
// Hermitian. make_hermitian (non-Hermitian input): G <- (G + G^H) / 2.
size_t gram_workspace_elems(int64_t m, int64_t n);
cudaError_t zgram(cudaStream_t s, int64_t K, int64_t m, int64_t n, const double2* X,
                  int64_t ldx, const double2* Y, int64_t ldy, double2* G, int64_t ldg,
                  bool hermitian, double2* ws, size_t ws_elems);
cudaError_t hermitian_part(cudaStream_t s, int64_t n, double2* G, int64_t ldg);

// Skinny product P = A * B for n <= 8 columns (Lanczos), split-K partials in ws.
size_t skinny_workspace_elems(int64_t M, int64_t n);
cudaError_t zgemm_skinny(cudaStream_t s, int64_t M, int64_t n, const double2* A, int64_t lda,
                         const double2* B, int64_t ldb, double2* P, int64_t ldp, double2* ws);

// -------------------------------------------------------- factorisations
// Upper Cholesky G = U^H U in place (n x n, ldg); *info (device) = 0 or the
// 1-based first failing pivot. dinv receives the inverses of the 64 x 64
// diagonal blocks of U (ceil(n/64) blocks of 64*64, column-major).
constexpr int kNB = 64;
cudaError_t potrf_upper(cudaStream_t s, int64_t n, double2* G, int64_t ldg, double2* dinv,
                        int* info);
// X <- X U^{-1} (X: m x n, ldx), U upper from potrf_upper with its dinv.
cudaError_t trsm_right_upper(cudaStream_t s, int64_t m, int64_t n, double2* X, int64_t ldx,
                             const double2* U, int64_t ldu, const double2* dinv,
                             const int* info);
// Y = U^{-1} (n x n, ld ldy, upper triangular) from potrf_upper's U and dinv;
// T: scratch of at least n^2 / 4 + n entries.
cudaError_t triangular_inverse(cudaStream_t s, int64_t n, const double2* U, int64_t ldu,
                               const double2* dinv, double2* Y, int64_t ldy, double2* T);
// *out (device) = max over the upper triangle of |U_ij - delta_ij|.
cudaError_t max_dev_identity(cudaStream_t s, int64_t n, const double2* U, int64_t ldu,
                             double* out);
// M = I, or M -= I with subtract (n x n, ld ldm).
cudaError_t set_identity(cudaStream_t s, int64_t n, double2* M, int64_t ldm, bool subtract);
// *out (device) = max over columns j of max_i |R_ij| / max_i |X_ij| (m x n
// blocks, |z| = max(|Re z|, |Im z|); a zero column of X counts 0 or +inf).
cudaError_t max_col_ratio(cudaStream_t s, int64_t m, int64_t n, const double2* R, int64_t ldr,
                          const double2* X, int64_t ldx, double* out);
// Strict lower triangle of the n x n M (ld ldm) set to zero.
cudaError_t zero_lower(cudaStream_t s, int64_t n, double2* M, int64_t ldm);
// G_ii += shift * trace(G) (device scalars only); used for the shifted pass.
cudaError_t add_trace_shift(cudaStream_t s, int64_t n, double2* G, int64_t ldg, double factor,
                            double* scratch);

// Grouped raster order of an nrow x ncol grid of output tiles: consecutive CTAs
// take `group` row blocks of one column tile, then the same row blocks of the
// next column tile, so the CTAs resident at one time read a few row blocks of
// the left operand and a few column tiles of the right one, and L2 serves each
// tile to the rest of the wave instead of DRAM. Bijective on [0, nrow ncol).
__device__ __forceinline__ void grouped_tile(unsigned id, unsigned nrow, unsigned ncol,
                                             unsigned group, unsigned& row, unsigned& col) {
  const unsigned per = group * ncol;
  const unsigned g = id / per;
  const unsigned first = g * group;
  const unsigned rg = min(group, nrow - first);
  const unsigned local = id - g * per;
  row = first + local % rg;
  col = local / rg;
}

// ------------------------------------------------------------ eigensolver
// Two-sided cyclic Jacobi with round-robin parallel ordering on the n x n
// Hermitian G (destroyed). Eigenvalues ascending into w (device), eigenvectors
// into Z (n x n, ldz). *sweeps_out (host) and the status.
struct JacobiWork {
  double2* Gw;       // n x n working copy (ld n)
  double2* Gw2;      // second buffer: rounds alternate between Gw and Gw2
  double2* Zw;       // n x n unsorted eigenvectors (ld n)
  double2* Zw2;      // n x n rotations of the FP64 stage
  double2* T;        // n x n product scratch
  float2* G32a;      // FP32 stage: two working copies and the eigenvectors
  float2* G32b;
  float2* Z32;
  float2* Rb = nullptr;  // blocked FP32 Jacobi: one 64 x 64 rotation per block pair
  size_t rb_elems = 0;
  double2* gram_ws;  // borrowed from the context (free while Jacobi runs)
  size_t gram_ws_elems;
  double2* dinv;     // borrowed: POTRF diagonal-block inverses and info
  int* info;
  double* params;    // 4 per pair
  double* red;       // reduction scratch
  double* host_red;  // pinned host scalars
  double* host_part = nullptr;  // pinned host: 512 doubles of partial sums
  int64_t nmax;
  int max_sweeps = 0;  // > 0: cap on every stage (sweeps, refinement steps)
  int* pairs = nullptr;   // index pairs the refinement could not separate (2 ints each)
  int* npairs = nullptr;  // their count (device)
  int* cl_idx = nullptr;  // clustered column indices, grouped by cluster (n ints)
  int* cl_off = nullptr;  // cluster offsets into cl_idx (n + 1 ints)
  // optional product for the FP64 refinement: P = op(X) B (op(X) = X, M x K, or
  // X^H for X of K x M), epilogue as for zgemm_nn; extended: the accurate
  // variant for products that cancel; null: CUDA-core FP64 products
  cudaError_t (*gemm)(void* ctx, int64_t M, int64_t K, const double2* X, int64_t ldx,
                      bool conj_trans, int64_t ncols, const double2* B, int64_t ldb,
                      const Epilogue& ep, bool extended) = nullptr;
  void* gemm_ctx = nullptr;
};
size_t jacobi_params_elems(int64_t n);
// float2 elements of JacobiWork::Rb for matrices up to order n
size_t jacobi_rot_elems(int64_t n);
constexpr int kMaxClusterPairs = 1 << 16;  // capacity of JacobiWork::pairs
size_t jacobi_red_elems();  // doubles of JacobiWork::red
// cluster_out (3 ints, may be null): [0] 1 if the pairs the FP64 refinement
// could not separate were finished cluster by cluster, [1] the largest cluster,
// [2] the number of clusters (or of recorded pairs when the full FP64 sweeps ran).
int jacobi_heev(cudaStream_t s, int64_t n, const double2* G, int64_t ldg, double* w, double2* Z,
                int64_t ldz, JacobiWork& wk, int* sweeps_out, int* fp64_sweeps_out = nullptr,
                int* cluster_out = nullptr);
// Batched small Jacobi (n <= 64) on `batch` column-major n x n matrices with
// stride n*n; eigenvalues ascending (w: batch x n), eigenvectors Z; *status
// (device) set to 1 when a sweep cap is hit.
// max_sweeps > 0 lowers the sweep cap (default 40).
cudaError_t jacobi_small_batched(cudaStream_t s, int n, int batch, const double2* G, double* w,
                                 double2* Z, int* status, int max_sweeps = 0);

// -------------------------------------------------------------- vector ops
cudaError_t copy_cols(cudaStream_t s, int64_t m, int64_t n, const double2* src, int64_t lds,
                      double2* dst, int64_t ldd);
cudaError_t gather_cols(cudaStream_t s, int64_t m, int64_t n, const double2* src, int64_t lds,
                        const int* perm, double2* dst, int64_t ldd);

// Lanczos with nvec simultaneous runs (block HEMV + per-run BLAS-1); writes
// bounds (b_sup, mu_1, mu_ne, norm_est) to the device array out4.
struct LanczosWork {
  double2* Q;        // 3 buffers of N x 8 (prev, cur, next/w)
  double2* ws;       // skinny GEMM workspace
  double* red;       // partial sums
  double* ab;        // alpha/beta per run and step: [2][8][kmax]
  double2* T;        // batch of k x k tridiagonal matrices as complex
  double* theta;     // batch x k
  double2* Z;        // batch x k x k
  double* out4;      // b_sup, mu_1, mu_ne, norm_est
  int* status;
  // optional replacement of the block product W = A Q (e.g. on the tensor
  // cores); nullptr: the FP64 skinny GEMM
  cudaError_t (*matmul)(void* ctx, const double2* Q, int64_t ldq, int nvec, double2* W,
                        int64_t ldw) = nullptr;
  void* matmul_ctx = nullptr;
};
cudaError_t lanczos_bounds(cudaStream_t s, int64_t N, const double2* A, int64_t lda,
                           const double2* Q0, int64_t ldq, int nvec, int k, int64_t ne,
                           LanczosWork& w);

}  // namespace chase
