// Batching layer: many independent HDG problems (different n, p, data) and
// several right-hand sides each, solved concurrently on one GPU.
//
// Every problem gets its own context and its own CUDA stream; a pool of host
// threads drives the contexts, so the set-up and the solves of different
// problems overlap on the device (each context keeps its PCG loop in one
// CUDA graph).  The batch is ordered with respect to the caller's stream by
// events.  Built only on the public C ABI of hdgmg.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <string>
#include <thread>
#include <vector>

#include "internal.h"

struct hdgmg_batch {
  std::vector<hdgmg_ctx*> ctx;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> done;
  cudaEvent_t start = nullptr;
  cudaStream_t user = nullptr;
  int device = 0;
  int nthreads = 1;
};

namespace {

hdgmg_status bfail(hdgmg_status st, const std::string& msg) {
  hdgmg::set_last_error(msg);
  return st;
}

// Run work(i) for every problem on a pool of host threads; returns the first
// failure (and its message) in problem order.
template <typename F>
hdgmg_status for_each_problem(hdgmg_batch* b, F work) {
  const int np = (int)b->ctx.size();
  std::vector<hdgmg_status> st(np, HDGMG_OK);
  std::vector<std::string> msg(np);
  if (cudaEventRecord(b->start, b->user) != cudaSuccess) return bfail(HDGMG_ECUDA, "event record");
  std::atomic<int> next{0};
  auto worker = [&] {
    cudaSetDevice(b->device);
    for (;;) {
      const int i = next.fetch_add(1);
      if (i >= np) break;
      if (cudaStreamWaitEvent(b->streams[i], b->start, 0) != cudaSuccess) {
        st[i] = HDGMG_ECUDA;
        msg[i] = "stream wait";
        continue;
      }
      st[i] = work(i);
      if (st[i] != HDGMG_OK) msg[i] = hdgmg_last_error();
      cudaEventRecord(b->done[i], b->streams[i]);
    }
  };
  const int nt = std::max(1, std::min(b->nthreads, np));
  std::vector<std::thread> pool;
  for (int t = 1; t < nt; ++t) pool.emplace_back(worker);
  worker();
  for (auto& th : pool) th.join();
  for (int i = 0; i < np; ++i) cudaStreamWaitEvent(b->user, b->done[i], 0);
  hdgmg_status first_err = HDGMG_OK, first_noconv = HDGMG_OK;
  std::string err_msg, noconv_msg;
  for (int i = 0; i < np; ++i) {
    if (st[i] == HDGMG_OK) continue;
    if (st[i] == HDGMG_ENOCONV) {
      if (first_noconv == HDGMG_OK) {
        first_noconv = st[i];
        noconv_msg = "problem " + std::to_string(i) + ": " + msg[i];
      }
    } else if (first_err == HDGMG_OK) {
      first_err = st[i];
      err_msg = "problem " + std::to_string(i) + ": " + msg[i];
    }
  }
  if (first_err != HDGMG_OK) return bfail(first_err, err_msg);
  if (first_noconv != HDGMG_OK) return bfail(first_noconv, noconv_msg);
  return HDGMG_OK;
}

}  // namespace

extern "C" {

void hdgmg_batch_destroy(hdgmg_batch* b) {
  if (!b) return;
  for (hdgmg_ctx* c : b->ctx) hdgmg_destroy(c);
  for (cudaStream_t s : b->streams)
    if (s) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->done)
    if (e) cudaEventDestroy(e);
  if (b->start) cudaEventDestroy(b->start);
  delete b;
}

hdgmg_status hdgmg_batch_create(hdgmg_batch** out, int32_t nprob, const hdgmg_problem* problems,
                                const hdgmg_opts* opts, int32_t nthreads, void* stream) {
  if (!out) return bfail(HDGMG_EINVAL, "batch pointer is NULL");
  *out = nullptr;
  if (nprob < 1 || !problems) return bfail(HDGMG_EINVAL, "need nprob >= 1 problems");
  // the contexts of a batch run concurrently: one L2 set-aside cannot hold all
  // of their operators, so none of them asks for persisting lines
  hdgmg_opts bo;
  if (opts)
    bo = *opts;
  else
    hdgmg_default_opts(&bo);
  bo.l2_persist_mb = 0;
  // the persistent cycle is one cooperative grid per context; the batch's
  // contexts run concurrently on their own streams, so they use the launched
  // cycle
  bo.pcycle = 0;
  hdgmg_batch* b = new hdgmg_batch();
  b->user = (cudaStream_t)stream;
  cudaGetDevice(&b->device);
  b->nthreads = nthreads > 0 ? nthreads : 8;
  if (cudaEventCreateWithFlags(&b->start, cudaEventDisableTiming) != cudaSuccess) {
    hdgmg_batch_destroy(b);
    return bfail(HDGMG_ECUDA, "event create");
  }
  for (int i = 0; i < nprob; ++i) {
    cudaStream_t s = nullptr;
    cudaEvent_t e = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      hdgmg_batch_destroy(b);
      return bfail(HDGMG_ECUDA, "stream/event create");
    }
    b->streams.push_back(s);
    b->done.push_back(e);
    hdgmg_ctx* c = nullptr;
    hdgmg_status st = hdgmg_create(&c, &problems[i], &bo, s);
    if (st != HDGMG_OK) {
      std::string m = "problem " + std::to_string(i) + ": " + hdgmg_last_error();
      hdgmg_batch_destroy(b);
      return bfail(st, m);
    }
    b->ctx.push_back(c);
  }
  *out = b;
  return HDGMG_OK;
}

hdgmg_status hdgmg_batch_setup(hdgmg_batch* b, const double* const* log_kappa) {
  if (!b || !log_kappa) return bfail(HDGMG_EINVAL, "NULL argument");
  // one synchronous autotuning pass per distinct (p, operator kind) first, on
  // an otherwise idle device, then the set-ups run concurrently
  if (cudaStreamSynchronize(b->user) != cudaSuccess) return bfail(HDGMG_ECUDA, "stream sync");
  std::vector<std::pair<int, int>> seen;
  for (size_t i = 0; i < b->ctx.size(); ++i) {
    int p = 0, ns = 0;
    hdgmg::condensation_kind(b->ctx[i], &p, &ns);
    if (std::find(seen.begin(), seen.end(), std::make_pair(p, ns)) != seen.end()) continue;
    seen.emplace_back(p, ns);
    hdgmg_status st = hdgmg::tune_condensation(b->ctx[i], log_kappa[i]);
    if (st != HDGMG_OK) return st;
  }
  return for_each_problem(b, [&](int i) { return hdgmg_setup(b->ctx[i], log_kappa[i]); });
}

hdgmg_status hdgmg_batch_solve(hdgmg_batch* b, int32_t nrhs, const double* const* f,
                               const double* const* g_D, double* const* lambda, double* const* u,
                               double* const* q, hdgmg_info* infos) {
  if (!b || !f || !lambda) return bfail(HDGMG_EINVAL, "NULL argument");
  return for_each_problem(b, [&](int i) {
    return hdgmg_solve(b->ctx[i], nrhs, f[i], g_D ? g_D[i] : nullptr, lambda[i], u ? u[i] : nullptr,
                       q ? q[i] : nullptr, infos ? &infos[i] : nullptr);
  });
}

hdgmg_status hdgmg_batch_context(hdgmg_batch* b, int32_t i, hdgmg_ctx** ctx) {
  if (!b || !ctx || i < 0 || i >= (int)b->ctx.size()) return bfail(HDGMG_EINVAL, "bad index");
  *ctx = b->ctx[i];
  return HDGMG_OK;
}

}  // extern "C"
