// Many independent solves at once (a sequence of related problems, e.g. the
// Hamiltonians of successive self-consistent-field steps, each warm-started
// from the previous Ritz vectors). Every problem keeps its own context and
// stream; host threads drive the solves so that the kernels of different
// problems overlap on the GPU, which small problems (N of a few thousand) need
// to fill 152 SMs. Results are those of chase_solve on each problem alone: the
// kernels are the same and every reduction has a fixed order.
#include <algorithm>
#include <atomic>
#include <numeric>
#include <thread>
#include <vector>

#include "ctx.cuh"

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
  // largest problems first (their solves are the longest): cost ~ N^2 (nev + nex)
  std::vector<int64_t> order(count);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
    const double ca = (double)ctxs[a]->N * ctxs[a]->N * ctxs[a]->ne;
    const double cb = (double)ctxs[b]->N * ctxs[b]->N * ctxs[b]->ne;
    return ca > cb;
  });
  int nt = threads > 0 ? threads : 8;
  nt = (int)std::min<int64_t>(nt, count);
  std::atomic<int64_t> next{0};
  auto worker = [&]() {
    for (;;) {
      const int64_t i = next.fetch_add(1);
      if (i >= count) return;
      const int64_t k = order[i];
      chase_ctx* c = ctxs[k];
      if (cudaSetDevice(c->device) != cudaSuccess) {
        status[k] = CHASE_ERR_CUDA;
        continue;
      }
      status[k] = chase_solve(c, A[k], lda[k], V[k], ldv[k], Q0 ? Q0[k] : nullptr,
                              ldq ? ldq[k] : 0, ritz[k], resid[k], stats ? &stats[k] : nullptr);
    }
  };
  std::vector<std::thread> pool;
  pool.reserve(nt);
  for (int t = 0; t < nt; ++t) pool.emplace_back(worker);
  for (auto& t : pool) t.join();
  for (int64_t k = 0; k < count; ++k)
    if (status[k] != CHASE_OK) return status[k];
  return CHASE_OK;
}
