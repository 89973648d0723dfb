// ps_batch.cu -- many independent 2-way / 3-way problems in one persistent
// launch, captured once per batch in a CUDA graph, and the autotuner that
// picks the kernel variant of that launch.
//
// Not in the paper (its unit of work is one large decomposed problem, §4).
// Small problems launched one by one leave most SMs idle (a 256-vector 2-way
// instance has 3 tiles of 128 x 128 for 152 SMs); the batched launch puts the
// tiles of every problem in one work queue (ps_mgemm.cu, batched_kernel).
#include "ps_internal.cuh"

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

namespace ps {

struct CachedBatch {
  cudaGraphExec_t exec = nullptr;
  void* mem = nullptr;  // S, n2 tables, problem and item arrays, counters
  int* counters = nullptr;
  int nprob = 0;
  int nitems = 0;
};

struct BatchState {
  std::map<uint64_t, CachedBatch> graphs;  // key: problems + pointers + variant
  std::map<uint64_t, int> tuned;           // key: shapes only -> variant code
};

namespace {

uint64_t fnv(uint64_t h, const void* p, size_t n) {
  const unsigned char* c = static_cast<const unsigned char*>(p);
  for (size_t i = 0; i < n; ++i) {
    h ^= c[i];
    h *= 1099511628211ull;
  }
  return h;
}

uint64_t shape_signature(const ps_problem* probs, int n) {
  uint64_t h = 1469598103934665603ull;
  for (int t = 0; t < n; ++t) {
    const int64_t f[4] = {probs[t].V.nv, probs[t].V.nf, probs[t].way, probs[t].out_dtype};
    h = fnv(h, f, sizeof(f));
  }
  return h;
}

// Everything a captured launch depends on: shapes, pointers, kernel variant
// and the wait limit (a kernel argument baked into the graph).
uint64_t full_signature(const ps_problem* probs, int n, int variant, unsigned long long wait_ns) {
  uint64_t h = shape_signature(probs, n);
  for (int t = 0; t < n; ++t) {
    const uintptr_t f[3] = {(uintptr_t)probs[t].V.data, (uintptr_t)probs[t].out,
                            (uintptr_t)probs[t].V.ld};
    h = fnv(h, f, sizeof(f));
  }
  h = fnv(h, &wait_ns, sizeof(wait_ns));
  return fnv(h, &variant, sizeof(variant));
}

// Variant stored for shape signature `sigs` in a JSON-lines autotune cache
// (the last matching line wins), or -1.
int cached_variant(const char* path, const char* sigs) {
  int best = -1;
  if (!path || !*path) return best;
  if (FILE* f = fopen(path, "r")) {
    char line[1024];
    while (fgets(line, sizeof(line), f)) {
      const char* p = strstr(line, sigs);
      const char* v = strstr(line, "\"variant\": ");
      if (p && v) best = atoi(v + 11);
    }
    fclose(f);
  }
  return best;
}

// candidate configurations of the autotuner: the TMA-fed kernel
// (ps_batch_tma.cu, code 3000), and the cp.async kernel with tile 128 (8 or
// 16 warps) or 64 x unroll depth 16, 8, 4, all packed adds (see
// mgemm_variant_code)
constexpr int kTmaVariant = 3000;
const int kVariants[10] = {kTmaVariant, 108, 116, 104, 1108, 1116, 1104, 2108, 2116, 2104};

bool known_variant(int v) {
  for (int k : kVariants)
    if (k == v) return true;
  return false;
}

bool is_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

ps_status check_problems(ps_ctx* h, const ps_problem* probs, int n) {
  if (!probs || n <= 0) return fail(h, PS_ERR_INVALID_ARG, "batched: %d problems", n);
  for (int t = 0; t < n; ++t) {
    const ps_problem& p = probs[t];
    const ps_matrix& V = p.V;
    if (p.way != 2 && p.way != 3)
      return fail(h, PS_ERR_INVALID_ARG, "problem %d: way %d", t, p.way);
    if (V.nv < p.way || V.nv > (1 << 20) || V.nf < 0 || V.nf > (1 << 30))
      return fail(h, PS_ERR_INVALID_ARG, "problem %d: nv=%lld nf=%lld", t, (long long)V.nv,
                  (long long)V.nf);
    if (V.dtype != PS_F32 || V.layout != PS_LAYOUT_FIELD_MAJOR || V.ld < V.nv || V.ld % 4 != 0)
      return fail(h, PS_ERR_INVALID_ARG,
                  "problem %d: batched problems need FP32 field-major input, ld %% 4 == 0", t);
    if (!p.out || (V.nf > 0 && (!V.data || ((uintptr_t)V.data % 16) != 0)))
      return fail(h, PS_ERR_INVALID_ARG, "problem %d: null or misaligned pointer", t);
    if ((p.way == 2 && p.out_dtype != PS_F32 && p.out_dtype != PS_F64) ||
        (p.way == 3 && p.out_dtype != PS_F32))
      return fail(h, PS_ERR_INVALID_ARG, "problem %d: out_dtype %d", t, p.out_dtype);
    if ((V.nf > 0 && !is_device(V.data)) || !is_device(p.out))
      return fail(h, PS_ERR_INVALID_ARG, "problem %d: batched buffers must be device memory", t);
  }
  return PS_OK;
}

int64_t tiles3_of_pivot(int nv, int j, int B) {
  const int64_t Tk = (nv + B - 1) / B;
  const int64_t nI = (j + B - 1) / B;
  const int64_t nK = (j + 1 < nv) ? (Tk - (j + 1) / B) : 0;
  return nI * nK;
}

// Build the work list and device state of one batch and capture its graph.
// stall: testing aid (ps_config.test_batched_stall): problem 0's per-vector
// sums target is raised by one block that does not exist, so the first
// dependency wait on it runs out after the handle's wait limit.
ps_status build_batch(ps_ctx* h, const ps_problem* probs, int n, int variant, CachedBatch* cb,
                      bool stall = false) {
  const int B = mgemm_variant_of(variant)->tile;
  std::vector<BatchProb> bp(n);
  size_t off_S = 0, off_n2 = 0;
  std::vector<size_t> oS(n), oN(n);
  for (int t = 0; t < n; ++t) {
    oS[t] = off_S;
    off_S += (size_t)round_up(probs[t].V.nv, 32);
    oN[t] = off_n2;
    if (probs[t].way == 3) off_n2 += (size_t)probs[t].V.nv * probs[t].V.nv;
  }
  // items: sums | 2-way tiles + n2 tiles | 3-way tiles; groups longest-first
  std::vector<BatchItem> sums, mid, tail;
  for (int t = 0; t < n; ++t) {
    const int nv = (int)probs[t].V.nv;
    const int nsb = (int)ceil_div(nv, 32);
    for (int b = 0; b < nsb; ++b) sums.push_back({t, BK_SUMS, b, 0});
    const int T = (int)ceil_div(nv, B);
    for (int I = 0; I < T; ++I)
      for (int J = I; J < T; ++J) mid.push_back({t, probs[t].way == 2 ? BK_TILE2 : BK_N2, I, J});
    if (probs[t].way == 3)
      for (int j = 0; j < nv; ++j) {
        const int64_t c = tiles3_of_pivot(nv, j, B);
        for (int64_t u = 0; u < c; ++u) tail.push_back({t, BK_TILE3, j, (int)u});
      }
  }
  auto by_cost = [&](const BatchItem& a, const BatchItem& b) {
    return probs[a.prob].V.nf > probs[b.prob].V.nf;
  };
  std::stable_sort(mid.begin(), mid.end(), by_cost);
  std::stable_sort(tail.begin(), tail.end(), by_cost);
  std::vector<BatchItem> items;
  items.reserve(sums.size() + mid.size() + tail.size());
  items.insert(items.end(), sums.begin(), sums.end());
  items.insert(items.end(), mid.begin(), mid.end());
  items.insert(items.end(), tail.begin(), tail.end());
  if (items.size() > 0x7fffffff) return fail(h, PS_ERR_INVALID_ARG, "batched: too many work items");

  const size_t bytes_S = round_up((int64_t)off_S * 8, 256);
  const size_t bytes_n2 = round_up((int64_t)off_n2 * 4, 256);
  const size_t bytes_p = round_up((int64_t)n * sizeof(BatchProb), 256);
  const size_t bytes_i = round_up((int64_t)items.size() * sizeof(BatchItem), 256);
  const size_t bytes_c = round_up((int64_t)(2 + 2 * n) * sizeof(int), 256);
  char* mem = nullptr;
  cudaError_t e = cudaMalloc(&mem, bytes_S + bytes_n2 + bytes_p + bytes_i + bytes_c);
  if (e != cudaSuccess) return cuda_fail(h, e, "batched state");
  cb->mem = mem;
  double* S = reinterpret_cast<double*>(mem);
  float* N2 = reinterpret_cast<float*>(mem + bytes_S);
  BatchProb* dprob = reinterpret_cast<BatchProb*>(mem + bytes_S + bytes_n2);
  BatchItem* ditems = reinterpret_cast<BatchItem*>(mem + bytes_S + bytes_n2 + bytes_p);
  int* counters = reinterpret_cast<int*>(mem + bytes_S + bytes_n2 + bytes_p + bytes_i);
  for (int t = 0; t < n; ++t) {
    const ps_problem& p = probs[t];
    BatchProb& q = bp[t];
    q.v = VF32{static_cast<const float*>(p.V.data), p.V.ld, (int)p.V.nv, (int)p.V.nf};
    q.S = S + oS[t];
    q.n2 = p.way == 3 ? N2 + oN[t] : nullptr;
    q.out = p.out;
    q.way = p.way;
    q.out_f64 = p.out_dtype == PS_F64;
    q.nsum_blocks = (int)ceil_div(p.V.nv, 32) + ((stall && t == 0) ? 1 : 0);
    const int64_t T = ceil_div(p.V.nv, B);
    q.n2_tiles = p.way == 3 ? (int)(T * (T + 1) / 2) : 0;
  }
  PS_CUDA_TRY(h, cudaMemcpy(dprob, bp.data(), n * sizeof(BatchProb), cudaMemcpyHostToDevice));
  PS_CUDA_TRY(h, cudaMemcpy(ditems, items.data(), items.size() * sizeof(BatchItem),
                            cudaMemcpyHostToDevice));
  cb->counters = counters;
  cb->nprob = n;
  cb->nitems = (int)items.size();

  // attributes are set outside the capture
  PS_CUDA_TRY(h, launch_batched(h, variant, dprob, n, ditems, 0, counters, 0));
  cudaStream_t cs;
  PS_CUDA_TRY(h, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaMemsetAsync(counters, 0, (2 + 2 * n) * sizeof(int), cs);
    launch_batched(h, variant, dprob, n, ditems, cb->nitems, counters, cs);
    e = cudaStreamEndCapture(cs, &g);
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&cb->exec, g, 0);
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cs);
  if (e != cudaSuccess) return cuda_fail(h, e, "batched graph capture");
  return PS_OK;
}

// The TMA-fed variant (every problem needs n_f >= 1): problem records with
// their tensor maps, (problem, 32-vector) sum blocks, and the work list
// [2-way tiles + n2 tiles][3-way items], each group longest (largest n_f)
// first.  stall: testing aid (ps_config.test_batched_stall): the first 3-way
// problem's n2 target is raised by one warp store that never comes.
ps_status build_batch_tma(ps_ctx* h, const ps_problem* probs, int n, CachedBatch* cb, bool stall = false) {
  constexpr int B = 128;
  std::vector<BatchProbTma> bp(n);
  size_t off_S = 0, off_n2 = 0;
  std::vector<size_t> oS(n), oN(n);
  for (int t = 0; t < n; ++t) {
    oS[t] = off_S;
    off_S += (size_t)round_up(probs[t].V.nv, 32);
    oN[t] = off_n2;
    if (probs[t].way == 3) off_n2 += (size_t)probs[t].V.nv * probs[t].V.nv;
  }
  std::vector<int2> sblk;
  std::vector<BatchItem> mid, tail;
  bool stalled = false;
  for (int t = 0; t < n; ++t) {
    const ps_problem& p = probs[t];
    const int nv = (int)p.V.nv;
    for (int b = 0; b < (int)ceil_div(nv, 32); ++b) sblk.push_back(make_int2(t, b));
    const int T = (int)ceil_div(nv, B);
    for (int I = 0; I < T; ++I)
      for (int J = I; J < T; ++J) mid.push_back({t, p.way == 2 ? BK_TILE2 : BK_N2, I, J});
    if (p.way == 3) {
      if (T >= 65536) return fail(h, PS_ERR_INVALID_ARG, "batched: nv too large for the 3-way item table");
      for (int j = 0; j < nv; ++j) {
        const int nI = (j + B - 1) / B, k0 = (j + 1) / B;
        if (j + 1 >= nv) continue;
        for (int I = 0; I < nI; ++I)
          for (int K = k0; K < T; ++K) tail.push_back({t, BK_TILE3, j, (I << 16) | K});
      }
    }
    if (!make_batch_prob_tma(&bp[t], static_cast<const float*>(p.V.data), p.V.nv, p.V.nf, p.V.ld))
      return fail(h, PS_ERR_CUDA, "batched: tensor map of problem %d", t);
    bp[t].way = p.way;
    bp[t].out_f64 = p.out_dtype == PS_F64;
    bp[t].out = p.out;
    bp[t].n2_target = p.way == 3 ? (int)((int64_t)T * (T + 1) / 2 * 16) : 0;
    if (stall && p.way == 3 && !stalled) {
      bp[t].n2_target += 1;
      stalled = true;
    }
  }
  auto by_cost = [&](const BatchItem& a, const BatchItem& b) { return probs[a.prob].V.nf > probs[b.prob].V.nf; };
  std::stable_sort(mid.begin(), mid.end(), by_cost);
  std::stable_sort(tail.begin(), tail.end(), by_cost);
  std::vector<BatchItem> items;
  items.reserve(mid.size() + tail.size());
  items.insert(items.end(), mid.begin(), mid.end());
  items.insert(items.end(), tail.begin(), tail.end());
  if (items.size() > 0x7fffffff || sblk.size() > 0x7fffffff)
    return fail(h, PS_ERR_INVALID_ARG, "batched: too many work items");

  const size_t bytes_S = round_up((int64_t)off_S * 8, 256);
  const size_t bytes_n2 = round_up((int64_t)off_n2 * 4, 256);
  const size_t bytes_p = round_up((int64_t)n * sizeof(BatchProbTma), 256);
  const size_t bytes_b = round_up((int64_t)sblk.size() * sizeof(int2), 256);
  const size_t bytes_i = round_up((int64_t)items.size() * sizeof(BatchItem), 256);
  const size_t bytes_c = round_up((int64_t)(2 + n) * sizeof(int), 256);
  char* mem = nullptr;
  cudaError_t e = cudaMalloc(&mem, bytes_S + bytes_n2 + bytes_p + bytes_b + bytes_i + bytes_c);
  if (e != cudaSuccess) return cuda_fail(h, e, "batched state");
  cb->mem = mem;
  double* S = reinterpret_cast<double*>(mem);
  float* N2 = reinterpret_cast<float*>(mem + bytes_S);
  char* q = mem + bytes_S + bytes_n2;
  BatchProbTma* dprob = reinterpret_cast<BatchProbTma*>(q);
  int2* dblk = reinterpret_cast<int2*>(q + bytes_p);
  BatchItem* ditems = reinterpret_cast<BatchItem*>(q + bytes_p + bytes_b);
  int* counters = reinterpret_cast<int*>(q + bytes_p + bytes_b + bytes_i);
  for (int t = 0; t < n; ++t) {
    bp[t].S = S + oS[t];
    bp[t].n2 = probs[t].way == 3 ? N2 + oN[t] : nullptr;
  }
  PS_CUDA_TRY(h, cudaMemcpy(dprob, bp.data(), n * sizeof(BatchProbTma), cudaMemcpyHostToDevice));
  PS_CUDA_TRY(h, cudaMemcpy(dblk, sblk.data(), sblk.size() * sizeof(int2), cudaMemcpyHostToDevice));
  PS_CUDA_TRY(h, cudaMemcpy(ditems, items.data(), items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice));
  cb->counters = counters;
  cb->nprob = n;
  cb->nitems = (int)items.size();

  // attributes are set outside the capture (an empty launch)
  PS_CUDA_TRY(h, launch_batched_tma(h, dprob, dblk, 0, ditems, 0, counters, 0));
  cudaStream_t cs;
  PS_CUDA_TRY(h, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaMemsetAsync(counters, 0, (2 + n) * sizeof(int), cs);
    launch_batched_tma(h, dprob, dblk, (int)sblk.size(), ditems, cb->nitems, counters, cs);
    e = cudaStreamEndCapture(cs, &g);
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&cb->exec, g, 0);
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cs);
  if (e != cudaSuccess) return cuda_fail(h, e, "batched graph capture");
  return PS_OK;
}

bool all_fields_nonempty(const ps_problem* probs, int n) {
  for (int t = 0; t < n; ++t)
    if (probs[t].V.nf < 1) return false;
  return true;
}

// Reads the launch's error flag; PS_ERR_TIMEOUT if a dependency wait ran out.
ps_status graph_status(ps_ctx* h, const CachedBatch& cb, cudaStream_t st) {
  int herr = 0;
  PS_CUDA_TRY(h, cudaMemcpyAsync(&herr, cb.counters + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
  PS_CUDA_TRY(h, cudaStreamSynchronize(st));
  if (herr) return fail(h, PS_ERR_TIMEOUT, "batched launch: a dependency wait timed out");
  return PS_OK;
}

ps_status run_graph(ps_ctx* h, const ps_problem* probs, int n, int variant, cudaStream_t st) {
  if (!h->batch) h->batch = new BatchState();
  if (h->batched_stall) {
    // one-off launch with the stalled dependency; not cached
    h->batched_stall = 0;
    h->cfg.test_batched_stall = 0;
    CachedBatch cb;
    ps_status s = variant == kTmaVariant ? build_batch_tma(h, probs, n, &cb, true)
                                         : build_batch(h, probs, n, variant, &cb, true);
    if (s == PS_OK) {
      const cudaError_t e = cudaGraphLaunch(cb.exec, st);
      s = e == cudaSuccess ? graph_status(h, cb, st) : cuda_fail(h, e, "cudaGraphLaunch");
    }
    cudaStreamSynchronize(st);
    if (cb.exec) cudaGraphExecDestroy(cb.exec);
    if (cb.mem) cudaFree(cb.mem);
    return s;
  }
  const uint64_t key = full_signature(probs, n, variant, h->wait_ns);
  auto it = h->batch->graphs.find(key);
  if (it == h->batch->graphs.end()) {
    CachedBatch cb;
    ps_status s = variant == kTmaVariant ? build_batch_tma(h, probs, n, &cb) : build_batch(h, probs, n, variant, &cb);
    if (s != PS_OK) {
      if (cb.exec) cudaGraphExecDestroy(cb.exec);
      if (cb.mem) cudaFree(cb.mem);
      return s;
    }
    it = h->batch->graphs.emplace(key, cb).first;
  }
  {
    ScopedTimer tm(h, "batched", st);
    PS_CUDA_TRY(h, cudaGraphLaunch(it->second.exec, st));
  }
  return graph_status(h, it->second, st);
}

// The TMA-fed kernel (every problem needs at least one field), else the
// configured cp.async variant.
int default_variant(ps_ctx* h, const ps_problem* probs, int n) {
  return all_fields_nonempty(probs, n) ? kTmaVariant : mgemm_variant_code(h);
}

}  // namespace

void batch_state_free(ps_ctx* h) {
  if (!h->batch) return;
  for (auto& kv : h->batch->graphs) {
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (kv.second.mem) cudaFree(kv.second.mem);
  }
  delete h->batch;
  h->batch = nullptr;
}

}  // namespace ps

using namespace ps;

extern "C" ps_status ps_metrics_batched(ps_handle h, const ps_problem* probs, int32_t n, int32_t mode,
                                        ps_stream stream) {
  if (!h) return fail(nullptr, PS_ERR_INVALID_ARG, "null handle");
  if (mode != PS_BATCH_PERSISTENT && mode != PS_BATCH_PER_INSTANCE)
    return fail(h, PS_ERR_INVALID_ARG, "batched mode %d", mode);
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != h->device) cudaSetDevice(h->device);
  ps_status s = check_problems(h, probs, n);
  if (s == PS_OK && wants_fp64(h))
    s = fail(h, PS_ERR_UNSUPPORTED, "ps_metrics_batched has no FP64 kernel (handle precision is PS_PATH_FP64)");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (s == PS_OK) {
    if (mode == PS_BATCH_PER_INSTANCE) {
      for (int t = 0; t < n && s == PS_OK; ++t) {
        if (probs[t].way == 2)
          s = ps_metrics_2way(h, &probs[t].V, PS_PATH_FP32, 0, probs[t].out, probs[t].out_dtype, stream);
        else
          s = ps_metrics_3way(h, &probs[t].V, 0, probs[t].V.nv, static_cast<float*>(probs[t].out),
                              stream);
      }
    } else {
      // the handle's own tuning, else the configured autotune cache, else
      // the default variant
      int variant = default_variant(h, probs, n);
      const uint64_t sig = shape_signature(probs, n);
      bool tuned = false;
      if (h->batch) {
        auto it = h->batch->tuned.find(sig);
        if (it != h->batch->tuned.end()) {
          variant = it->second;
          tuned = true;
        }
      }
      if (!tuned && !h->cache_path.empty()) {
        char sigs[32];
        snprintf(sigs, sizeof(sigs), "%016llx", (unsigned long long)sig);
        const int v = cached_variant(h->cache_path.c_str(), sigs);
        if (known_variant(v) && (v != kTmaVariant || all_fields_nonempty(probs, n))) variant = v;
      }
      s = run_graph(h, probs, n, variant, st);
    }
  }
  if (prev >= 0 && prev != h->device) cudaSetDevice(prev);
  return s;
}

extern "C" ps_status ps_autotune_batched(ps_handle h, const ps_problem* probs, int32_t n,
                                         const char* cache_path, char* choice, int32_t choice_len,
                                         ps_stream stream) {
  if (!h) return fail(nullptr, PS_ERR_INVALID_ARG, "null handle");
  ps_status s = check_problems(h, probs, n);
  if (s != PS_OK) return s;
  if (!h->batch) h->batch = new BatchState();
  const uint64_t sig = shape_signature(probs, n);
  char sigs[32];
  snprintf(sigs, sizeof(sigs), "%016llx", (unsigned long long)sig);
  // the call's cache path, else the handle's configured one; a cache hit
  // skips the measurement
  if (!cache_path && !h->cache_path.empty()) cache_path = h->cache_path.c_str();
  int best = cached_variant(cache_path, sigs);
  if (!known_variant(best)) best = -1;
  std::string detail;
  if (best < 0) {
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    PS_CUDA_TRY(h, cudaEventCreate(&e0));
    PS_CUDA_TRY(h, cudaEventCreate(&e1));
    float best_ms = 1e30f;
    for (int vc : kVariants) {
      if (vc == kTmaVariant && !all_fields_nonempty(probs, n)) continue;
      s = run_graph(h, probs, n, vc, st);  // build + warm up
      if (s != PS_OK) break;
      float ms_min = 1e30f;
      for (int rep = 0; rep < 2 && s == PS_OK; ++rep) {
        cudaEventRecord(e0, st);
        s = run_graph(h, probs, n, vc, st);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms_min = std::min(ms_min, ms);
      }
      char buf[64];
      snprintf(buf, sizeof(buf), "%s\"%d\": %.3f", detail.empty() ? "" : ", ", vc, ms_min);
      detail += buf;
      if (ms_min < best_ms) {
        best_ms = ms_min;
        best = vc;
      }
      // keep only the graph of the winner so far
      for (auto it = h->batch->graphs.begin(); it != h->batch->graphs.end();) {
        if (it->first == full_signature(probs, n, vc, h->wait_ns) && vc != best) {
          cudaGraphExecDestroy(it->second.exec);
          cudaFree(it->second.mem);
          it = h->batch->graphs.erase(it);
        } else {
          ++it;
        }
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != PS_OK) return s;
    if (cache_path) {
      if (FILE* f = fopen(cache_path, "a")) {
        fprintf(f, "{\"shape_signature\": \"%s\", \"problems\": %d, \"variant\": %d, \"ms\": {%s}}\n",
                sigs, n, best, detail.c_str());
        fclose(f);
      }
    }
  }
  h->batch->tuned[sig] = best;
  if (choice && choice_len > 0) {
    const int shape = best / 1000;
    if (best == kTmaVariant)
      snprintf(choice, (size_t)choice_len, "TMA-fed pipeline, tile 128 x 128 (16 warps), 64-field slices%s",
               detail.empty() ? " (cached)" : "");
    else
      snprintf(choice, (size_t)choice_len, "cp.async tile %d x %d (%d warps), %s add, %d-step unroll%s",
               shape == 1 ? 64 : 128, shape == 1 ? 64 : 128, shape == 1 ? 2 : (shape == 2 ? 16 : 8),
               (best / 100) % 10 ? "packed f32x2" : "scalar", best % 100, detail.empty() ? " (cached)" : "");
  }
  return PS_OK;
}
