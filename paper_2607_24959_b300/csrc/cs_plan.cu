// cs_plan.cu -- execution plans for the fused forward + adjoint path.
//
// A plan is made once for one ragged batch and its output buffers:
//  * instances are bucketed by (nv bucket, rows per lane MT), so an instance
//    with few rows runs in a kernel whose per-warp shared-memory slice (and so
//    its occupancy) fits it, and a small-nv instance does not pay for a large
//    padded nv;
//  * inside a bucket the warps claim instances from a device counter in
//    descending cost order (m nv^2 + nv^3), so the longest solves start first
//    and the tail is made of the cheapest ones;
//  * warps per block is tuned per bucket by timing the candidates on the
//    plan's own data (autotuner; results cached per device and bucket);
//  * the bucket kernels are captured into one CUDA graph as parallel branches
//    (counter resets included), so a replay is one cudaGraphLaunch and a
//    bucket that finishes early frees its SMs to the others.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "contact_solve.h"
#include "cs_host.h"
#include "cs_cta.cuh"

namespace cs {

namespace {

struct Bucket {
  int nvb = 0, mt = 0, n = 0, wpb = 2;
  bool cta = false;      // one CTA per instance (nv > 32 or m > 256)
  int nv_max = 0, m_max = 0;
  double cost = 0.0;
  float tuned_ms = 0.f;
  int32_t* d_order = nullptr;
  int32_t* d_counter = nullptr;
};

// (device ordinal, nv bucket, MT) -> tuned warps per block
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, std::pair<int, float>> g_tune;

int current_device() {
  int d = 0;
  cudaGetDevice(&d);
  return d;
}

}  // namespace

}  // namespace cs

struct cs_plan {
  int device = 0;
  cs_options opt{};
  csk::Params base{};
  std::vector<cs::Bucket> buckets;
  void* d_mem = nullptr;
  cudaStream_t side[8] = {};
  int n_side = 0;
  cudaEvent_t ev_fork = nullptr;
  cudaEvent_t ev_join[8] = {};
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace cs {
namespace {

cudaError_t launch_bucket(const cs_plan* p, const Bucket& b, int wpb, cudaStream_t s) {
  csk::Params P = p->base;
  P.n_work = b.n;
  P.order = b.d_order;
  P.counter = b.d_counter;
  cudaError_t e = cudaMemsetAsync(b.d_counter, 0, sizeof(int32_t), s);
  if (e != cudaSuccess) return e;
  LaunchCfg cfg;
  cfg.warps_per_block = wpb;
  if (b.cta) return launch_cta(csk::MODE_FUSED, b.nv_max, b.m_max, P, s, nullptr);
  return launch_warp(csk::MODE_FUSED, b.nvb, 32 * b.mt, P, cfg, s, nullptr);
}

void destroy_plan(cs_plan* p) {
  if (!p) return;
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  for (int i = 0; i < p->n_side; ++i) {
    if (p->side[i]) cudaStreamDestroy(p->side[i]);
    if (p->ev_join[i]) cudaEventDestroy(p->ev_join[i]);
  }
  if (p->ev_fork) cudaEventDestroy(p->ev_fork);
  if (p->d_mem) cudaFree(p->d_mem);
  delete p;
}

int autotune_bucket(cs_plan* p, Bucket& b, cudaStream_t s) {
  static const int cand[] = {1, 2, 4, 8};
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return cuda_error(cudaGetLastError(), "autotune");
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_error(cudaGetLastError(), "autotune");
  }
  float best = 1e30f;
  int best_w = 2;
  int rc = CS_OK;
  for (int w : cand) {
    cudaError_t e = launch_bucket(p, b, w, s);  // warm-up
    if (e != cudaSuccess) { rc = cuda_error(e, "autotune launch"); break; }
    cudaEventRecord(e0, s);
    const int reps = 3;
    for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch_bucket(p, b, w, s);
    cudaEventRecord(e1, s);
    if (e != cudaSuccess) { rc = cuda_error(e, "autotune launch"); break; }
    e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) { rc = cuda_error(e, "autotune sync"); break; }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    ms /= reps;
    if (ms < best) {
      best = ms;
      best_w = w;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != CS_OK) return rc;
  b.wpb = best_w;
  b.tuned_ms = best;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[std::make_tuple(p->device, b.nvb, b.mt)] = {best_w, best};
  return CS_OK;
}

int capture_graph(cs_plan* p) {
  cudaStream_t s0 = p->side[0];
  cudaError_t e = cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_error(e, "graph capture begin");
  cudaError_t first = cudaSuccess;
  const int nb = (int)p->buckets.size();
  if (nb > 1) {
    first = cudaEventRecord(p->ev_fork, s0);
    for (int i = 1; i < nb && first == cudaSuccess; ++i)
      first = cudaStreamWaitEvent(p->side[i], p->ev_fork, 0);
  }
  for (int i = 0; i < nb && first == cudaSuccess; ++i)
    first = launch_bucket(p, p->buckets[i], p->buckets[i].wpb, p->side[i]);
  if (first == cudaErrorInvalidConfiguration) first = cudaErrorInvalidValue;
  for (int i = 1; i < nb && first == cudaSuccess; ++i) {
    first = cudaEventRecord(p->ev_join[i], p->side[i]);
    if (first == cudaSuccess) first = cudaStreamWaitEvent(s0, p->ev_join[i], 0);
  }
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(s0, &g);
  if (first != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_error(first, "graph capture");
  }
  if (e != cudaSuccess) return cuda_error(e, "graph capture end");
  p->graph = g;
  e = cudaGraphInstantiate(&p->exec, g, 0);
  if (e != cudaSuccess) return cuda_error(e, "graph instantiate");
  return CS_OK;
}

}  // namespace
}  // namespace cs

using namespace cs;

extern "C" {

int cs_plan_create_fused(const cs_batch* batch, const cs_options* opt, const cs_inst* inst_host,
                         const float* g, float* a, float* dqfrc, float* daref, float* dJ,
                         int32_t* status, int32_t* iters, int32_t flags, void* stream,
                         cs_plan** out) {
  return cs_plan_create_fused_theta(batch, opt, inst_host, g, a, dqfrc, daref, dJ, nullptr,
                                    nullptr, status, iters, flags, stream, out);
}

int cs_plan_create_fused_theta(const cs_batch* batch, const cs_options* opt,
                               const cs_inst* inst_host, const float* g, float* a, float* dqfrc,
                               float* daref, float* dJ, float* dM, float* dD, int32_t* status,
                               int32_t* iters, int32_t flags, void* stream, cs_plan** out) {
  if (!out) return set_error(CS_EINVAL, "out must not be NULL");
  *out = nullptr;
  int rc = check_batch_shapes(batch, opt);
  if (rc != CS_OK) return rc;
  if (batch->n > 0 && (!inst_host || !g || !a || !dqfrc || !status || !iters ||
                       (batch->m_max > 0 && (!daref || !dJ))))
    return set_error(CS_EINVAL, "inst_host, g and the outputs must not be NULL");
  cs_plan* p = new cs_plan();
  p->device = current_device();
  p->opt = *opt;
  p->base = make_params(batch, opt);
  p->base.g = g;
  p->base.a = a;
  p->base.dqfrc = dqfrc;
  p->base.daref = daref;
  p->base.dJ = dJ;
  p->base.dM = dM;
  p->base.dD = batch->m_max > 0 ? dD : nullptr;
  p->base.status = status;
  p->base.iters = iters;
  cudaStream_t s = (cudaStream_t)stream;

  // bucket the instances (shapes outside the kernels go to the smallest
  // bucket, where the kernel marks them CS_ST_BADSHAPE)
  // key (nv bucket, MT) for warp buckets; (-1, rows per thread) for the CTA
  // buckets, whose shared memory is sized from the bucket's own maxima
  std::map<std::pair<int, int>, std::vector<std::pair<double, int32_t>>> groups;
  std::map<std::pair<int, int>, std::pair<int, int>> maxima;
  for (int32_t i = 0; i < batch->n; ++i) {
    const cs_inst& e = inst_host[i];
    std::pair<int, int> key;
    const bool bad = e.nv < 1 || e.m < 0 || e.nv > batch->nv_max || e.m > batch->m_max;
    if (bad) {
      key = {3, 1};
    } else if (uses_warp_kernel(e.nv, e.m)) {
      key = {nv_bucket(e.nv), mt_bucket(e.m)};
    } else {
      // CTA buckets by nv (multiples of 32) and rows per thread
      key = {-((e.nv + 31) / 32), cta_rows_per_thread(e.m)};
    }
    const double nv = e.nv > 0 ? e.nv : 1, m = e.m > 0 ? e.m : 0;
    groups[key].push_back({m * nv * nv + nv * nv * nv, i});
    auto& mx = maxima[key];
    if (!bad) {
      mx.first = std::max(mx.first, e.nv);
      mx.second = std::max(mx.second, e.m);
    }
  }
  size_t total = 0;
  for (auto& kv : groups) {
    Bucket b;
    b.nvb = kv.first.first;
    b.mt = kv.first.second;
    b.n = (int)kv.second.size();
    b.cta = b.nvb < 0;
    b.nv_max = std::max(1, maxima[kv.first].first);
    b.m_max = maxima[kv.first].second;
    if (b.cta) b.wpb = csk::kCtaWarps;
    std::stable_sort(kv.second.begin(), kv.second.end(),
                     [](const std::pair<double, int32_t>& x, const std::pair<double, int32_t>& y) {
                       return x.first > y.first;
                     });
    for (auto& c : kv.second) b.cost += c.first;
    p->buckets.push_back(b);
    total += ((size_t)b.n * sizeof(int32_t) + 255) & ~(size_t)255;
    total += 256;
  }
  std::sort(p->buckets.begin(), p->buckets.end(),
            [](const Bucket& x, const Bucket& y) { return x.cost > y.cost; });
  for (const auto& b : p->buckets) {
    if (b.cta && cta_smem_bytes(b.nv_max, b.m_max) > device_smem_optin()) {
      const size_t need = cta_smem_bytes(b.nv_max, b.m_max);
      destroy_plan(p);
      return set_error(CS_EUNSUPPORTED,
                       "instances with nv up to %d and m up to %d need %zu bytes of shared "
                       "memory per CTA (limit %zu)",
                       b.nv_max, b.m_max, need, device_smem_optin());
    }
  }
  if ((int)p->buckets.size() > 8) {
    destroy_plan(p);
    return set_error(CS_EUNSUPPORTED, "more than 8 kernel buckets");
  }
  cudaError_t e = cudaSuccess;
  if (total) {
    e = cudaMalloc(&p->d_mem, total);
    if (e != cudaSuccess) {
      destroy_plan(p);
      return set_error(CS_ENOMEM, "plan buffers: %s", cudaGetErrorString(e));
    }
    char* cur = (char*)p->d_mem;
    std::vector<int32_t> h;
    for (auto& b : p->buckets) {
      const auto& lst = groups[{b.nvb, b.mt}];
      h.clear();
      for (auto& c : lst) h.push_back(c.second);
      b.d_counter = (int32_t*)cur;
      cur += 256;
      b.d_order = (int32_t*)cur;
      cur += ((size_t)b.n * sizeof(int32_t) + 255) & ~(size_t)255;
      e = cudaMemcpy(b.d_order, h.data(), h.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
      if (e != cudaSuccess) break;
    }
    if (e != cudaSuccess) {
      destroy_plan(p);
      return cuda_error(e, "plan upload");
    }
  }
  // launch geometry: explicit, tuned, cached or default
  for (auto& b : p->buckets) {
    if (b.cta) continue;
    if (opt->warps_per_block > 0) {
      b.wpb = opt->warps_per_block;
      continue;
    }
    if (flags & CS_PLAN_AUTOTUNE) {
      rc = autotune_bucket(p, b, s);
      if (rc != CS_OK) {
        destroy_plan(p);
        return rc;
      }
      continue;
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(std::make_tuple(p->device, b.nvb, b.mt));
    b.wpb = (it != g_tune.end()) ? it->second.first : 2;
  }
  if (flags & CS_PLAN_GRAPH) {
    p->n_side = std::max<int>(1, (int)p->buckets.size());
    for (int i = 0; i < p->n_side; ++i) {
      e = cudaStreamCreateWithFlags(&p->side[i], cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_join[i], cudaEventDisableTiming);
      if (e != cudaSuccess) break;
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      destroy_plan(p);
      return cuda_error(e, "plan streams");
    }
    // the graph reads buffers the caller may still be writing on `stream`
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      destroy_plan(p);
      return cuda_error(e, "plan sync");
    }
    rc = capture_graph(p);
    if (rc != CS_OK) {
      destroy_plan(p);
      return rc;
    }
  }
  *out = p;
  return CS_OK;
}

int cs_plan_launch(cs_plan* p, void* stream) {
  if (!p) return set_error(CS_EINVAL, "plan must not be NULL");
  cudaStream_t s = (cudaStream_t)stream;
  if (p->exec) {
    cudaError_t e = cudaGraphLaunch(p->exec, s);
    return e == cudaSuccess ? CS_OK : cuda_error(e, "cs_plan_launch graph");
  }
  for (auto& b : p->buckets) {
    cudaError_t e = launch_bucket(p, b, b.wpb, s);
    if (e != cudaSuccess) return cuda_error(e, "cs_plan_launch");
  }
  return CS_OK;
}

int cs_plan_describe(const cs_plan* p, cs_plan_info* info) {
  if (!p || !info) return set_error(CS_EINVAL, "plan and info must not be NULL");
  memset(info, 0, sizeof(*info));
  info->n_kernels = (int32_t)p->buckets.size();
  info->graph = p->exec != nullptr;
  for (size_t i = 0; i < p->buckets.size() && i < 8; ++i) {
    const Bucket& b = p->buckets[i];
    info->nv_bucket[i] = b.nvb;
    info->rows_per_lane[i] = b.mt;
    info->instances[i] = b.n;
    info->warps_per_block[i] = b.wpb;
    info->tuned_ms[i] = b.tuned_ms;
    info->cta[i] = b.cta ? 1 : 0;
    if (b.cta) info->nv_bucket[i] = b.nv_max;
  }
  return CS_OK;
}

void cs_plan_destroy(cs_plan* p) { destroy_plan(p); }

int cs_autotune_cache_dump(char* buf, size_t len) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  std::string s;
  char line[128];
  for (auto& kv : g_tune) {
    snprintf(line, sizeof(line), "%d %d %d %d %.6f\n", std::get<0>(kv.first),
             std::get<1>(kv.first), std::get<2>(kv.first), kv.second.first, kv.second.second);
    s += line;
  }
  if (buf && len > 0) {
    size_t k = std::min(len - 1, s.size());
    memcpy(buf, s.data(), k);
    buf[k] = 0;
  }
  return (int)s.size();
}

int cs_autotune_cache_load(const char* text) {
  if (!text) return set_error(CS_EINVAL, "text must not be NULL");
  std::lock_guard<std::mutex> lk(g_tune_mu);
  int n = 0;
  const char* cur = text;
  while (*cur) {
    int dev, nvb, mt, wpb;
    float ms;
    int used = 0;
    if (sscanf(cur, "%d %d %d %d %f%n", &dev, &nvb, &mt, &wpb, &ms, &used) != 5) break;
    if (wpb >= 1 && wpb <= 8 && nv_bucket(nvb) == nvb && mt_bucket(32 * mt) == mt) {
      g_tune[std::make_tuple(dev, nvb, mt)] = {wpb, ms};
      ++n;
    }
    cur += used;
    while (*cur == '\n' || *cur == ' ' || *cur == '\r') ++cur;
  }
  return n;
}

}  // extern "C"
