// Many independent solves at once (a sequence of related problems, e.g. the
// Hamiltonians of successive self-consistent-field steps, each warm-started
// from the previous Ritz vectors).
//
// The problems advance through Alg. 2 in lockstep, phase by phase: a pool of
// host threads runs every problem's Lanczos start, its degree/sort/CondEst
// step, and its QR, Rayleigh-Ritz, residual and locking step on the problem's
// own context and stream (so small problems overlap on the GPU); the filter
// phase of all problems that are in the reduced-precision mode (and live on
// one device) runs as one CUDA graph of grouped tensor-core launches, one
// launch per degree step covering every such problem's tiles, and so does the
// filter phase of all problems in the FP64 mode with the tensor-core FP64
// products (per degree step one launch slicing every problem's operand
// columns into digits and one product launch). Problems in the FP64 mode with
// the CUDA-core products filter with their own launches. Each problem's
// arithmetic, and so its results, are those of chase_solve on it alone: the
// grouped launches run every tile and column exactly as the per-problem
// launches do, and every reduction has a fixed order.
#include <algorithm>
#include <atomic>
#include <map>
#include <memory>
#include <numeric>
#include <thread>
#include <vector>

#include "ctx.cuh"

namespace {

using chase::SolveState;

// f(k) for every k of idx on up to nt host threads; each thread makes the
// problem's device current first.
template <typename F>
void run_parallel(const std::vector<int64_t>& idx, int nt, chase_ctx* const* ctxs, int32_t* status,
                  F f) {
  if (idx.empty()) return;
  nt = (int)std::min<int64_t>(nt, (int64_t)idx.size());
  std::atomic<size_t> next{0};
  auto worker = [&]() {
    for (;;) {
      const size_t i = next.fetch_add(1);
      if (i >= idx.size()) return;
      const int64_t k = idx[i];
      if (cudaSetDevice(ctxs[k]->device) != cudaSuccess) {
        status[k] = CHASE_ERR_CUDA;
        continue;
      }
      f(k);
    }
  };
  if (nt <= 1) {
    worker();
    return;
  }
  std::vector<std::thread> pool;
  pool.reserve(nt);
  for (int t = 0; t < nt; ++t) pool.emplace_back(worker);
  for (auto& t : pool) t.join();
}

// The grouped filter phase of the problems in idx (all on `device`, all in
// the reduced-precision mode) on the batch stream s.
int grouped_filter(int device, cudaStream_t s, const std::vector<int64_t>& idx,
                   std::vector<std::unique_ptr<SolveState>>& S, chase::MixedGroupTable& tab) {
  if (cudaSetDevice(device) != cudaSuccess) return CHASE_CUDA_FAIL();
  const size_t n = idx.size();
  std::vector<std::vector<double>> al(n), be(n);
  std::vector<chase::MixedGroupItem> items(n);
  for (size_t i = 0; i < n; ++i) {
    SolveState& st = *S[idx[i]];
    chase_ctx* c = st.c;
    const int64_t nact = c->ne - st.locked;
    const int32_t* degs = st.degs.data() + st.locked;
    chase::cheb_coefficients(degs[nact - 1], st.cc, st.ee, st.mu_1, c->p.scaled_filter != 0, al[i],
                             be[i]);
    items[i] = chase::MixedGroupItem{c->N, st.A, st.lda, st.C + st.locked * st.ldv, st.ldv,
                                     nact, degs, st.cc, al[i].data(), be[i].data(), &c->mw};
  }
  if (chase::mixed_group_reserve(tab, chase::mixed_group_entries((int)n, items.data())) !=
      cudaSuccess)
    return CHASE_ERR_OOM;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return CHASE_CUDA_FAIL();
  cudaEventRecord(e0, s);
  const long long l0 = chase::launch_count();
  const int rc = chase::mixed_filter_grouped(s, (int)n, items.data(), tab, nullptr);
  const long long nl = chase::launch_count() - l0;
  cudaEventRecord(e1, s);
  float ms = 0.f;
  if (cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != CHASE_OK) return rc;
  for (size_t i = 0; i < n; ++i) {
    SolveState& st = *S[idx[i]];
    // the shared launches are charged to every problem in the group
    st.st.ms_filter += ms;
    st.launches += nl;
    chase::solve_count_filter(st);
  }
  return CHASE_OK;
}

// The grouped filter phase of the problems in idx (all on `device`, all in the
// FP64 mode with the tensor-core products) on the batch stream s.
int grouped_fp64_filter(int device, cudaStream_t s, const std::vector<int64_t>& idx,
                        std::vector<std::unique_ptr<SolveState>>& S, chase::OzakiGroupTable& tab) {
  if (cudaSetDevice(device) != cudaSuccess) return CHASE_CUDA_FAIL();
  const size_t n = idx.size();
  std::vector<std::vector<double>> al(n), be(n);
  std::vector<chase::OzakiGroupItem> items(n);
  for (size_t i = 0; i < n; ++i) {
    SolveState& st = *S[idx[i]];
    chase_ctx* c = st.c;
    if (!c->oz_a_valid) return CHASE_ERR_INVALID_ARG;  // A's digits come with solve_begin
    const int64_t nact = c->ne - st.locked;
    const int32_t* degs = st.degs.data() + st.locked;
    chase::cheb_coefficients(degs[nact - 1], st.cc, st.ee, st.mu_1, c->p.scaled_filter != 0, al[i],
                             be[i]);
    items[i] = chase::OzakiGroupItem{c->N, st.C + st.locked * st.ldv, st.ldv, c->W, c->N, nact,
                                     degs, st.cc, al[i].data(), be[i].data(), &c->ow};
  }
  if (chase::ozaki_group_reserve(tab, chase::ozaki_group_entries((int)n, items.data())) !=
      cudaSuccess)
    return CHASE_ERR_OOM;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return CHASE_CUDA_FAIL();
  cudaEventRecord(e0, s);
  const long long l0 = chase::launch_count();
  const int rc = chase::ozaki_filter_grouped(s, (int)n, items.data(), tab, nullptr);
  const long long nl = chase::launch_count() - l0;
  cudaEventRecord(e1, s);
  float ms = 0.f;
  if (cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != CHASE_OK) return rc;
  for (size_t i = 0; i < n; ++i) {
    SolveState& st = *S[idx[i]];
    st.st.ms_filter += ms;
    st.launches += nl;
    chase::solve_count_filter(st);
  }
  return CHASE_OK;
}

}  // namespace

extern "C" int chase_solve_batch(int64_t count, chase_ctx* const* ctxs, const chase_c128* const* A,
                                 const int64_t* lda, chase_c128* const* V, const int64_t* ldv,
                                 const chase_c128* const* Q0, const int64_t* ldq,
                                 double* const* ritz, double* const* resid, chase_stats* stats,
                                 int32_t* status, int32_t threads) {
  if (count < 0 || (count > 0 && (!ctxs || !A || !lda || !V || !ldv || !ritz || !resid || !status)))
    return CHASE_ERR_INVALID_ARG;
  if (count == 0) return CHASE_OK;
  for (int64_t k = 0; k < count; ++k) {
    if (!ctxs[k]) return CHASE_ERR_INVALID_ARG;
    for (int64_t j = 0; j < k; ++j)
      if (ctxs[j] == ctxs[k]) return CHASE_ERR_INVALID_ARG;  // a context is not shareable
  }
  int dev0 = 0;
  cudaGetDevice(&dev0);
  // largest problems first in every phase (their work is the longest): N^2 (nev + nex)
  std::vector<int64_t> order(count);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
    const double ca = (double)ctxs[a]->N * ctxs[a]->N * ctxs[a]->ne;
    const double cb = (double)ctxs[b]->N * ctxs[b]->N * ctxs[b]->ne;
    return ca > cb;
  });
  const int nt = threads > 0 ? threads : 8;
  std::vector<std::unique_ptr<SolveState>> S(count);
  for (int64_t k = 0; k < count; ++k) {
    S[k] = std::make_unique<SolveState>();
    status[k] = CHASE_OK;
  }
  run_parallel(order, nt, ctxs, status, [&](int64_t k) {
    status[k] = chase::solve_begin(*S[k], ctxs[k], reinterpret_cast<const double2*>(A[k]), lda[k],
                                   reinterpret_cast<double2*>(V[k]), ldv[k],
                                   reinterpret_cast<const double2*>(Q0 ? Q0[k] : nullptr),
                                   ldq ? ldq[k] : 0, ritz[k], resid[k]);
  });
  std::map<int, cudaStream_t> batch_stream;  // one per device holding grouped problems
  std::map<int, chase::MixedGroupTable> tables;
  std::map<int, chase::OzakiGroupTable> oz_tables;
  auto alive = [&]() {
    std::vector<int64_t> a;
    for (int64_t k : order)
      if (status[k] == CHASE_OK && chase::solve_active(*S[k])) a.push_back(k);
    return a;
  };
  for (std::vector<int64_t> act = alive(); !act.empty(); act = alive()) {
    run_parallel(act, nt, ctxs, status, [&](int64_t k) { status[k] = chase::solve_prepare(*S[k]); });
    // groups per (device, precision tier): reduced precision, FP64 on the tensor cores
    std::map<std::pair<int, int>, std::vector<int64_t>> grouped;
    std::vector<int64_t> own;
    for (int64_t k : act) {
      if (status[k] != CHASE_OK) continue;
      if (S[k]->mixed) grouped[{ctxs[k]->device, 0}].push_back(k);
      else if (ctxs[k]->p.fp64_tensor) grouped[{ctxs[k]->device, 1}].push_back(k);
      else own.push_back(k);
    }
    for (auto& g : grouped) {
      if (g.second.size() == 1) {  // nothing to share
        own.push_back(g.second[0]);
        continue;
      }
      const int dev = g.first.first;
      cudaStream_t& bs = batch_stream[dev];
      if (!bs) {
        if (cudaSetDevice(dev) != cudaSuccess ||
            cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking) != cudaSuccess) {
          for (int64_t k : g.second) status[k] = CHASE_ERR_CUDA;
          continue;
        }
      }
      const int rc = g.first.second == 0
                         ? grouped_filter(dev, bs, g.second, S, tables[dev])
                         : grouped_fp64_filter(dev, bs, g.second, S, oz_tables[dev]);
      if (rc != CHASE_OK)
        for (int64_t k : g.second) status[k] = rc;
    }
    run_parallel(own, nt, ctxs, status, [&](int64_t k) { status[k] = chase::solve_filter(*S[k]); });
    std::vector<int64_t> fin;
    for (int64_t k : act)
      if (status[k] == CHASE_OK) fin.push_back(k);
    run_parallel(fin, nt, ctxs, status, [&](int64_t k) { status[k] = chase::solve_complete(*S[k]); });
  }
  std::vector<int64_t> done;
  for (int64_t k : order)
    if (status[k] == CHASE_OK) done.push_back(k);
  run_parallel(done, nt, ctxs, status, [&](int64_t k) {
    status[k] = chase::solve_end(*S[k], stats ? &stats[k] : nullptr);
  });
  for (auto& b : batch_stream) {
    cudaSetDevice(b.first);
    if (b.second) cudaStreamDestroy(b.second);
  }
  for (auto& t : tables) {
    cudaSetDevice(t.first);
    chase::mixed_group_free(t.second);
  }
  for (auto& t : oz_tables) {
    cudaSetDevice(t.first);
    chase::ozaki_group_free(t.second);
  }
  S.clear();
  cudaSetDevice(dev0);
  for (int64_t k = 0; k < count; ++k)
    if (status[k] != CHASE_OK) return status[k];
  return CHASE_OK;
}
