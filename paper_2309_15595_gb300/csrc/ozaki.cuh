// FP64-accurate complex GEMM on BF16 tensor cores (digit slicing with exact
// chunked accumulation), see ozaki.cu.
#pragma once

#include "common.cuh"

namespace chase {

struct OzakiWork {
  void* Ad = nullptr;           // 6 digit planes of [Ar | Ai], N x 2Np each (BF16)
  void* Bd = nullptr;           // 6 digit planes of the right operand, brows x 2Np each
  int* ea = nullptr;            // row exponents of A
  int* eb = nullptr;            // column exponents of the right operand
  unsigned long long* amax = nullptr;
  double2* diag = nullptr;      // diagonal of A (applied exactly, outside the digits)
  int* err = nullptr;
  void* maps = nullptr;         // TMA tensor maps (pinned host)
  const void* A_ready = nullptr;  // A whose digits are in Ad
  void* Ld = nullptr;           // digit planes of a general left operand (N x n^2 products)
  size_t l_elems = 0;
  int* el = nullptr;            // row exponents of the general left operand
  int64_t l_M = 0, l_K = 0;     // layout of the planes in Ld (0: not yet written)
  int64_t N = 0, ne = 0, Np = 0, brows = 0;
};

int64_t ozaki_np(int64_t N);
cudaError_t ozaki_alloc(OzakiWork& w, int64_t N, int64_t ne);
void ozaki_free(OzakiWork& w);
// Digits and row exponents of A (must precede ozaki_gemm with this A).
cudaError_t ozaki_prepare_a(cudaStream_t s, const double2* A, int64_t lda, OzakiWork& w);
// P = A * B[:, j0:ncols_end] with the FP64 epilogue `ep` (EPI_STORE, EPI_FILTER or
// EPI_RESID; for EPI_RESID the partials are per 32-row tile, ceil(N/32) per
// column, indexed by absolute column). Y, X, theta, partial use absolute columns.
cudaError_t ozaki_gemm(cudaStream_t s, int64_t ncols_end, int64_t j0, const double2* B,
                       int64_t ldb, const Epilogue& ep, OzakiWork& w);
// P = op(X) * B for the N x n^2 products: op(X) = X (M x K, column-major) or,
// with conj_trans, X^H for X of K x M; B is K x ncols. No diagonal split. The
// epilogue uses absolute columns 0 .. ncols of B, X, Y. K <= N, ncols <= ne.
// extended: also keep the digit pairs of level 8 (26 instead of 21 products;
// the dropped pairs weigh 2^-58 instead of 2^-50 of the row and column scales),
// for products whose result cancels almost completely.
cudaError_t ozaki_gemm_general(cudaStream_t s, int64_t M, int64_t K, const double2* X,
                               int64_t ldx, bool conj_trans, int64_t ncols, const double2* B,
                               int64_t ldb, const Epilogue& ep, OzakiWork& w,
                               bool extended = false);
// X (M x K, column-major, M <= N) <- the digits it has as the left
// operand of ozaki_gemm_general (rows scaled by powers of two, six digits), so
// that such a product takes X exactly: a change of at most 2^-49 of each row's
// scale, leaving the row maxima (and so the scales) as they were except when a
// maximum rounds up to the next power of two.
cudaError_t ozaki_round_left(cudaStream_t s, int64_t M, int64_t K, double2* X, int64_t ldx,
                             OzakiWork& w);
// *out (device) = the largest row exponent e of the last general product's left
// operand (rows scaled by 2^-e to |x| < 1/2): bounds its digit-sliced error.
cudaError_t ozaki_left_exp_max(cudaStream_t s, int64_t M, OzakiWork& w, int* out);
// Reads and clears the device error flag; returns a chase_status.
int ozaki_check(cudaStream_t s, OzakiWork& w);

// One problem of a grouped FP64-accurate filter (several problems' filters in
// the same kernel launches): Eq. 1 on V[:, 0:ncols] with W as the ping-pong
// buffer, the steps the per-problem filter takes with ozaki_gemm. A's digits
// must be in w (ozaki_prepare_a).
struct OzakiGroupItem {
  int64_t N;
  double2* V;
  int64_t ldv;
  double2* W;
  int64_t ldw;
  int64_t ncols;
  const int32_t* degs;  // host, even, ascending
  double c;
  const double* al;     // host, dmax + 1 coefficients (al[i], be[i] of step i)
  const double* be;
  OzakiWork* w;
};
// Per-step, per-problem launch entries (device + pinned host) of the product
// and of the digit slicing.
struct OzakiGroupTable {
  void* dev = nullptr;
  void* host = nullptr;
  void* sdev = nullptr;
  void* shost = nullptr;
  size_t capacity = 0;  // entries of each
};
// Entries a grouped filter of these items needs (sum of their largest degrees).
size_t ozaki_group_entries(int count, const OzakiGroupItem* items);
cudaError_t ozaki_group_reserve(OzakiGroupTable& t, size_t entries);
void ozaki_group_free(OzakiGroupTable& t);
// All items' filters on stream s as one CUDA graph: per degree step i one
// launch that slices the operand columns of every problem whose largest
// degree is >= i and one product launch over all their tiles. Each problem's
// result equals that of its own filter with ozaki_gemm, bit for bit.
// Synchronises s. *launches (may be null) receives the number of launches.
int ozaki_filter_grouped(cudaStream_t s, int count, const OzakiGroupItem* items,
                         OzakiGroupTable& t, int* launches);

}  // namespace chase
