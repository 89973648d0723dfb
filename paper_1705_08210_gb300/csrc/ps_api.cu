// ps_api.cu -- the extern "C" boundary declared in include/ps.h.
//
// Argument checking, pointer-kind detection (device vs host), host staging
// through the handle's workspace, and dispatch to the kernels.
#include "ps_internal.cuh"

#include <algorithm>
#include <cstdarg>
#include <cstdlib>
#include <cstring>
#include <initializer_list>
#include <mutex>
#include <new>
#include <vector>

namespace ps {

static std::mutex g_err_mu;
static std::string g_last_error;

ps_status fail(ps_ctx* h, ps_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (h) h->last_error = buf;
  std::lock_guard<std::mutex> g(g_err_mu);
  g_last_error = buf;
  return st;
}

ps_status cuda_fail(ps_ctx* h, cudaError_t e, const char* where) {
  cudaGetLastError();  // clear a sticky launch error where possible
  if (e == cudaErrorMemoryAllocation)
    return fail(h, PS_ERR_OOM, "%s: %s", where, cudaGetErrorString(e));
  return fail(h, PS_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

void* ws_get(ps_ctx* h, WsSlot slot, size_t bytes) {
  Workspace& w = h->ws;
  if (bytes == 0) bytes = 256;
  if (w.bytes[slot] >= bytes) return w.ptr[slot];
  if (w.ptr[slot]) {
    cudaDeviceSynchronize();  // the old buffer may still be in use by queued work
    cudaFree(w.ptr[slot]);
    w.ptr[slot] = nullptr;
    w.bytes[slot] = 0;
  }
  const size_t sz = (size_t)round_up((int64_t)bytes, 256);
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, sz);
  if (e != cudaSuccess) {
    cudaGetLastError();
    fail(h, PS_ERR_OOM, "workspace slot %d: cudaMalloc(%zu) failed: %s", (int)slot, sz,
         cudaGetErrorString(e));
    return nullptr;
  }
  w.ptr[slot] = p;
  w.bytes[slot] = sz;
  return p;
}

int* async_err_word(ps_ctx* h) {
  if (!h->async_err_dev) {
    void* p = nullptr;
    cudaError_t e = cudaHostAlloc(&p, 256, cudaHostAllocMapped);
    if (e != cudaSuccess) {
      cudaGetLastError();
      fail(h, PS_ERR_OOM, "cudaHostAlloc(mapped error word): %s", cudaGetErrorString(e));
      return nullptr;
    }
    void* d = nullptr;
    e = cudaHostGetDevicePointer(&d, p, 0);
    if (e != cudaSuccess) {
      cudaGetLastError();
      cudaFreeHost(p);
      fail(h, PS_ERR_CUDA, "cudaHostGetDevicePointer(mapped error word): %s", cudaGetErrorString(e));
      return nullptr;
    }
    h->async_err_host = static_cast<int*>(p);
    *(volatile int*)h->async_err_host = 0;
    h->async_err_dev = static_cast<int*>(d);
  }
  return h->async_err_dev;
}

ScopedTimer::ScopedTimer(ps_ctx* h_, const char* name, cudaStream_t st_) : h(h_), st(st_) {
  if (!h || !h->timing) return;
  TimingRec r{name, nullptr, nullptr};
  if (cudaEventCreate(&r.a) != cudaSuccess || cudaEventCreate(&r.b) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  cudaEventRecord(r.a, st);
  h->trecs.push_back(r);
  idx = (int)h->trecs.size() - 1;
}

ScopedTimer::~ScopedTimer() {
  if (idx >= 0) cudaEventRecord(h->trecs[idx].b, st);
}

static void timing_clear(ps_ctx* h) {
  for (auto& r : h->trecs) {
    cudaEventSynchronize(r.b);
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  h->trecs.clear();
}

ps_status apply_config(ps_ctx* h, const ps_config* user) {
  ps_config c;
  ps_config_init(&c);
  if (user) c = *user;
  auto bad = [h](const char* field, long long v) {
    return fail(h, PS_ERR_INVALID_ARG, "ps_config.%s = %lld is outside its range", field, v);
  };
  auto one_of = [](int v, std::initializer_list<int> ok) {
    for (int x : ok)
      if (v == x) return true;
    return false;
  };
  if (!one_of(c.precision, {PS_PATH_FP32, PS_PATH_FP64})) return bad("precision", c.precision);
  if (!one_of(c.debug_checks, {0, 1})) return bad("debug_checks", c.debug_checks);
  if (c.wait_limit_ns < 1000 || c.wait_limit_ns > 60000000000LL) return bad("wait_limit_ns", c.wait_limit_ns);
  if (!one_of(c.mgemm_feed, {0, 1, 2})) return bad("mgemm_feed", c.mgemm_feed);
  if (!one_of(c.mgemm3_feed, {0, 1, 2})) return bad("mgemm3_feed", c.mgemm3_feed);
  if (!one_of(c.mgemm_tile, {0, 64, 128})) return bad("mgemm_tile", c.mgemm_tile);
  if (!one_of(c.mgemm_warps, {0, 8, 16})) return bad("mgemm_warps", c.mgemm_warps);
  if (!one_of(c.mgemm_unroll, {0, 4, 8, 16})) return bad("mgemm_unroll", c.mgemm_unroll);
  if (!one_of(c.mgemm_add, {0, 1, 2, 3})) return bad("mgemm_add", c.mgemm_add);
  if (c.mgemm_band < 0 || c.mgemm_band > 64) return bad("mgemm_band", c.mgemm_band);
  if (!one_of(c.tma_slice, {0, 16, 32, 64})) return bad("tma_slice", c.tma_slice);
  if (!one_of(c.tma_unroll, {0, 8, 16, 32})) return bad("tma_unroll", c.tma_unroll);
  if (!one_of(c.tma_stages, {0, 3, 4, 6})) return bad("tma_stages", c.tma_stages);
  if (!one_of(c.tma_schedule, {0, 1, 2})) return bad("tma_schedule", c.tma_schedule);
  if (c.tma_meet < 0 || c.tma_meet > 1 << 20) return bad("tma_meet", c.tma_meet);
  if (!one_of(c.mgemm3_schedule, {0, 1, 2})) return bad("mgemm3_schedule", c.mgemm3_schedule);
  if (!one_of(c.thermo_tile_m, {0, 128, 256})) return bad("thermo_tile_m", c.thermo_tile_m);
  if (c.thermo_meet_kb < -1 || c.thermo_meet_kb > 1 << 20) return bad("thermo_meet_kb", c.thermo_meet_kb);
  if (!one_of(c.test_batched_stall, {0, 1})) return bad("test_batched_stall", c.test_batched_stall);
  if (!one_of(c.mgemm_narrow, {0, 1, 2})) return bad("mgemm_narrow", c.mgemm_narrow);
  if (c.tma_lookahead < 0 || c.tma_lookahead > 7) return bad("tma_lookahead", c.tma_lookahead);
  if (!one_of(c.host_direct, {0, 1})) return bad("host_direct", c.host_direct);
  h->cache_path = c.autotune_cache ? c.autotune_cache : "";
  c.autotune_cache = c.autotune_cache ? h->cache_path.c_str() : nullptr;
  h->cfg = c;
  h->wait_ns = (unsigned long long)c.wait_limit_ns;
  h->mgemm_feed_tma = c.mgemm_feed != 2;
  h->mgemm3_feed_tma = c.mgemm3_feed != 2;
  h->mgemm_tile = c.mgemm_tile == 64 ? 64 : 128;
  h->mgemm_warps = c.mgemm_warps;
  h->mgemm_ku = c.mgemm_unroll ? c.mgemm_unroll : 8;
  h->mgemm_packed_add = c.mgemm_add != 2;
  h->mgemm_add = c.mgemm_add;
  h->mgemm_band = c.mgemm_band ? c.mgemm_band : 16;
  h->mgemm_tma_bk = c.tma_slice;
  h->mgemm_tma_ku = c.tma_unroll;
  h->mgemm_tma_stages = c.tma_stages ? c.tma_stages : 4;
  h->mgemm_tma_dynamic = c.tma_schedule != 2;
  h->mgemm_tma_sync = c.tma_schedule == 2 ? c.tma_meet : 0;
  h->mgemm3_dynamic = c.mgemm3_schedule != 2;
  h->thermo_tile_m = c.thermo_tile_m;
  h->thermo_sync_kb = c.thermo_meet_kb == 0 ? 960 : (c.thermo_meet_kb < 0 ? 0 : c.thermo_meet_kb);
  h->batched_stall = c.test_batched_stall;
  h->mgemm_narrow = c.mgemm_narrow;
  h->tma_lookahead = c.tma_lookahead;
  h->host_direct = c.host_direct;
  return PS_OK;
}

namespace {

// Memory kind of a caller pointer.
enum PtrKind { PK_DEVICE, PK_HOST };

ps_status ptr_kind(ps_ctx* h, const void* p, PtrKind* kind) {
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *kind = PK_HOST;  // unregistered pageable host memory on older runtimes
    return PS_OK;
  }
  switch (a.type) {
    case cudaMemoryTypeDevice:
      if (a.device != h->device)
        return fail(h, PS_ERR_INVALID_ARG, "device pointer belongs to device %d, handle uses %d",
                    a.device, h->device);
      *kind = PK_DEVICE;
      return PS_OK;
    case cudaMemoryTypeManaged:
      *kind = PK_DEVICE;
      return PS_OK;
    default:
      *kind = PK_HOST;
      return PS_OK;
  }
}

// bytes per stored element (a 32-bit word of 32 fields for PS_B1)
size_t dtype_size(int32_t dt) { return dt == PS_F64 ? 8 : (dt == PS_U8 ? 1 : 4); }
int out2_mode(int32_t out_dtype) {
  return out_dtype == PS_F64 ? OUT2_C2_F64 : (out_dtype == PS_U8 ? OUT2_C2_U8 : OUT2_C2_F32);
}

// Elements spanned by the matrix in its own layout.
int64_t matrix_span(const ps_matrix& V) {
  if (V.nv == 0 || V.nf == 0) return 0;
  if (V.dtype == PS_B1) return (V.nv - 1) * V.ld + ceil_div(V.nf, 32);
  if (V.layout == PS_LAYOUT_FIELD_MAJOR) return (V.nf - 1) * V.ld + V.nv;
  return (V.nv - 1) * V.ld + V.nf;
}

ps_status check_matrix(ps_ctx* h, const ps_matrix* V, int64_t min_nv) {
  if (!V) return fail(h, PS_ERR_INVALID_ARG, "null matrix descriptor");
  if (V->dtype != PS_F32 && V->dtype != PS_F64 && V->dtype != PS_B1)
    return fail(h, PS_ERR_INVALID_ARG, "dtype %d is not PS_F32/PS_F64/PS_B1", V->dtype);
  if (V->layout != PS_LAYOUT_FIELD_MAJOR && V->layout != PS_LAYOUT_VECTOR_MAJOR)
    return fail(h, PS_ERR_INVALID_ARG, "layout %d is not a ps_layout", V->layout);
  if (V->dtype == PS_B1 && V->layout != PS_LAYOUT_VECTOR_MAJOR)
    return fail(h, PS_ERR_INVALID_ARG, "PS_B1 needs PS_LAYOUT_VECTOR_MAJOR");
  if (V->nv < min_nv) return fail(h, PS_ERR_INVALID_ARG, "nv=%lld < %lld", (long long)V->nv, (long long)min_nv);
  if (V->nf < 0) return fail(h, PS_ERR_INVALID_ARG, "nf=%lld < 0", (long long)V->nf);
  if (V->nv > (int64_t)1 << 30 || V->nf > (int64_t)1 << 30)
    return fail(h, PS_ERR_INVALID_ARG, "nv or nf exceeds 2^30");
  const int64_t need =
      V->dtype == PS_B1 ? ceil_div(V->nf, 32) : (V->layout == PS_LAYOUT_FIELD_MAJOR ? V->nv : V->nf);
  if (V->ld < need || V->ld < 1)
    return fail(h, PS_ERR_INVALID_ARG, "ld=%lld smaller than the contiguous extent %lld",
                (long long)V->ld, (long long)need);
  if (V->nv > 0 && V->nf > 0 && !V->data) return fail(h, PS_ERR_INVALID_ARG, "null data pointer");
  return PS_OK;
}

struct Guard {  // makes the handle's device current for the call
  int prev = -1;
  explicit Guard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~Guard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

// Resolve V to a device-resident descriptor (copying host data into the
// workspace) and build the FP32 field-major view the kernels read.
struct Prepared {
  ps_matrix dev;   // device-resident version of the caller matrix
  VF32 f32;        // FP32 field-major view (may alias dev)
  double* S = nullptr;
  bool host_input = false;
};

ps_status prepare(ps_ctx* h, const ps_matrix& V, cudaStream_t st, bool need_f32, Prepared* P,
                  bool need_sums = true) {
  P->dev = V;
  PtrKind k = PK_DEVICE;
  if (V.nv > 0 && V.nf > 0) {
    ps_status s = ptr_kind(h, V.data, &k);
    if (s != PS_OK) return s;
  }
  if (k == PK_HOST) {
    const size_t bytes = (size_t)matrix_span(V) * dtype_size(V.dtype);
    void* d = ws_get(h, WS_INPUT, bytes);
    if (!d) return PS_ERR_OOM;
    if (bytes) PS_CUDA_TRY(h, cudaMemcpyAsync(d, V.data, bytes, cudaMemcpyHostToDevice, st));
    P->dev.data = d;
    P->host_input = true;
  }
  if (h->cfg.debug_checks) {
    // the paper's precondition v >= 0 (Section 2.1), and finite values
    auto* bad = static_cast<unsigned long long*>(ws_get(h, WS_AUX2, 256));
    if (!bad) return PS_ERR_OOM;
    PS_CUDA_TRY(h, launch_count_invalid(P->dev, bad, st));
    unsigned long long nbad = 0;
    PS_CUDA_TRY(h, cudaMemcpyAsync(&nbad, bad, sizeof(nbad), cudaMemcpyDeviceToHost, st));
    PS_CUDA_TRY(h, cudaStreamSynchronize(st));
    if (nbad)
      return fail(h, PS_ERR_INVALID_ARG, "debug check: %llu input values are negative, NaN or infinite", nbad);
  }
  if (need_sums) {
    P->S = static_cast<double*>(ws_get(h, WS_SUMS, (size_t)std::max<int64_t>(V.nv, 1) * 8));
    if (!P->S) return PS_ERR_OOM;
    ScopedTimer tm(h, "vector_sums", st);
    PS_CUDA_TRY(h, launch_vector_sums(P->dev, P->S, st));
  }
  if (!need_f32) return PS_OK;
  const bool direct = V.dtype == PS_F32 && V.layout == PS_LAYOUT_FIELD_MAJOR && V.ld % 4 == 0 &&
                      ((uintptr_t)P->dev.data % 16) == 0;
  if (direct) {
    P->f32 = VF32{static_cast<const float*>(P->dev.data), V.ld, (int)V.nv, (int)V.nf};
  } else {
    const int64_t ldp = round_up(V.nv, 4);
    float* d = static_cast<float*>(ws_get(h, WS_PACKED, (size_t)std::max<int64_t>(V.nf * ldp, 1) * 4));
    if (!d) return PS_ERR_OOM;
    {
      ScopedTimer tm(h, "pack", st);
      PS_CUDA_TRY(h, launch_pack_f32(P->dev, d, ldp, st));
    }
    P->f32 = VF32{d, ldp, (int)V.nv, (int)V.nf};
  }
  return PS_OK;
}

// FP64 field-major operand of the FP64 kernel: the caller's matrix when it
// already is one, else an exact widening / transpose into the workspace.
ps_status fp64_operand(ps_ctx* h, const ps_matrix* V, const Prepared& P, cudaStream_t st, const double** X,
                       int64_t* ld) {
  if (V->dtype == PS_F64 && V->layout == PS_LAYOUT_FIELD_MAJOR) {
    *X = static_cast<const double*>(P.dev.data);
    *ld = V->ld;
    return PS_OK;
  }
  const int64_t ldp = round_up(V->nv, 4);
  double* d = static_cast<double*>(ws_get(h, WS_PACKED, (size_t)std::max<int64_t>(V->nf * ldp, 1) * 8));
  if (!d) return PS_ERR_OOM;
  PS_CUDA_TRY(h, launch_pack_f64(P.dev, d, ldp, st));
  *X = d;
  *ld = ldp;
  return PS_OK;
}

// Device address of host memory that is pinned or registered with CUDA
// (device-mapped), else null.
void* mapped_host(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// Output buffer: caller device memory, or workspace staging for host memory.
struct OutBuf {
  void* dev = nullptr;
  void* user = nullptr;
  size_t bytes = 0;
  bool host = false;
};

ps_status resolve_out(ps_ctx* h, void* user, size_t bytes, WsSlot slot, OutBuf* o) {
  o->user = user;
  o->bytes = bytes;
  PtrKind k;
  ps_status s = ptr_kind(h, user, &k);
  if (s != PS_OK) return s;
  if (k == PK_DEVICE) {
    o->dev = user;
    return PS_OK;
  }
  o->host = true;
  o->dev = ws_get(h, slot, bytes);
  return o->dev ? PS_OK : PS_ERR_OOM;
}

// A pipeline wait of the TMA-fed kernel timed out (2 s) in this call, if it
// synchronised, or in an earlier asynchronous call on the handle: report it
// once.
ps_status take_async_error(ps_ctx* h) {
  if (h->async_err_host && *(volatile int*)h->async_err_host) {
    *(volatile int*)h->async_err_host = 0;
    return fail(h, PS_ERR_TIMEOUT,
                "a min-product pipeline wait timed out in this or an earlier asynchronous call on this "
                "handle; that call's output is incomplete");
  }
  return PS_OK;
}

ps_status finish(ps_ctx* h, const OutBuf& o, bool any_host, cudaStream_t st) {
  if (o.host && o.bytes)
    PS_CUDA_TRY(h, cudaMemcpyAsync(o.user, o.dev, o.bytes, cudaMemcpyDeviceToHost, st));
  if (any_host) {
    PS_CUDA_TRY(h, cudaStreamSynchronize(st));
    const ps_status s = take_async_error(h);
    if (s != PS_OK) return s;
  }
  PS_CUDA_TRY(h, cudaGetLastError());
  return PS_OK;
}

// Percentile P of the nonzero entries into the handle's select state.
ps_status run_percentile(ps_ctx* h, const VF32& v, cudaStream_t st, SelectState** state) {
  auto* sel = static_cast<unsigned char*>(ws_get(h, WS_AUX1, 2048 * 8 + 256));
  if (!sel) return PS_ERR_OOM;
  *state = reinterpret_cast<SelectState*>(sel + 2048 * 8);
  ScopedTimer tm(h, "quantize", st);
  PS_CUDA_TRY(h, launch_percentile_nonzero(h, v, 0.999, *state,
                                           reinterpret_cast<unsigned long long*>(sel), st));
  return PS_OK;
}

// Thermometer path of ps_metrics_2way (quantize, encode, tensor-core GEMM).
ps_status thermo_2way(ps_ctx* h, const VF32& v, int levels, void* out, int out_mode, cudaStream_t st) {
  SelectState* sel = nullptr;
  ps_status s = run_percentile(h, v, st, &sel);
  if (s != PS_OK) return s;
  const int nv_pad = (int)round_up(v.nv, 256);
  const int64_t Kpad = thermo_kpad(v.nf, levels);
  uint8_t* T = static_cast<uint8_t*>(ws_get(h, WS_QUANT, (size_t)nv_pad * Kpad));
  int* SQ = static_cast<int*>(ws_get(h, WS_AUX2, (size_t)nv_pad * sizeof(int)));
  int* err = static_cast<int*>(ws_get(h, WS_AUX3, 256));
  if (!T || !SQ || !err) return PS_ERR_OOM;
  PS_CUDA_TRY(h, cudaMemsetAsync(err, 0, sizeof(int), st));
  unsigned* sync = reinterpret_cast<unsigned*>(err + 32);
  {
    ScopedTimer tm(h, "thermo_encode", st);
    PS_CUDA_TRY(h, launch_thermo_encode(v, levels, sel, T, Kpad, nv_pad, SQ, st));
  }
  {
    ScopedTimer tm(h, "thermo_gemm", st);
    PS_CUDA_TRY(h, launch_thermo_gemm(h, T, Kpad, v.nv, nv_pad, SQ, out, out_mode, err, sync, st));
  }
  int herr = 0;
  PS_CUDA_TRY(h, cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  PS_CUDA_TRY(h, cudaStreamSynchronize(st));
  if (herr) return fail(h, PS_ERR_TIMEOUT, "tensor-core pipeline wait timed out");
  return PS_OK;
}

// Bit-packed 0/1 input on the tensor cores: the bits are the operand (the
// thermometer code of two levels), SQ the popcounts; exact.
ps_status binary_2way(ps_ctx* h, const ps_matrix& Vdev, void* out, int out_mode, cudaStream_t st) {
  const int nv = (int)Vdev.nv;
  const int nv_pad = (int)round_up(nv, 256);
  const int64_t Kpad = round_up(std::max<int64_t>(Vdev.nf, 1), 128);
  uint8_t* T = static_cast<uint8_t*>(ws_get(h, WS_QUANT, (size_t)nv_pad * Kpad));
  int* SQ = static_cast<int*>(ws_get(h, WS_AUX2, (size_t)nv_pad * sizeof(int)));
  int* err = static_cast<int*>(ws_get(h, WS_AUX3, 256));
  if (!T || !SQ || !err) return PS_ERR_OOM;
  PS_CUDA_TRY(h, cudaMemsetAsync(err, 0, sizeof(int), st));
  unsigned* sync = reinterpret_cast<unsigned*>(err + 32);
  {
    ScopedTimer tm(h, "b1_encode", st);
    PS_CUDA_TRY(h, launch_b1_encode(static_cast<const uint32_t*>(Vdev.data), Vdev.ld, nv, Vdev.nf, T, Kpad,
                                    nv_pad, SQ, st));
  }
  {
    ScopedTimer tm(h, "thermo_gemm", st);
    PS_CUDA_TRY(h, launch_thermo_gemm(h, T, Kpad, nv, nv_pad, SQ, out, out_mode, err, sync, st));
  }
  int herr = 0;
  PS_CUDA_TRY(h, cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  PS_CUDA_TRY(h, cudaStreamSynchronize(st));
  if (herr) return fail(h, PS_ERR_TIMEOUT, "tensor-core pipeline wait timed out");
  return PS_OK;
}

int key_bits_for(int nv) {
  int b = 1;
  while ((1 << b) < nv) ++b;
  return b;
}

// Run the thresholded kernel over `blk` (3 ints per block), sort the hits,
// write the first `capacity` and the total count.  Synchronous.
ps_status threshold_blocks(ps_ctx* h, const VF32& v, const double* S, const int* perm,
                           const std::vector<int>& blk, float tau, ps_triple* out, int64_t capacity,
                           int64_t* count, cudaStream_t st) {
  const int nv = v.nv;
  const float* n2 = static_cast<const float*>(h->ws.ptr[WS_N2]);
  const int64_t nblocks = (int64_t)blk.size() / 3;
  int* dblk = static_cast<int*>(ws_get(h, WS_BLOCKS, std::max<size_t>(blk.size(), 1) * sizeof(int)));
  if (!dblk) return PS_ERR_OOM;
  if (nblocks)
    PS_CUDA_TRY(h, cudaMemcpyAsync(dblk, blk.data(), blk.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  const int bits = key_bits_for(nv);
  int64_t cap = std::max<int64_t>({capacity, (int64_t)1 << 20, h->thresh_cap});
  int64_t total = 0;
  unsigned long long* counter = static_cast<unsigned long long*>(ws_get(h, WS_AUX3, 256));
  if (!counter) return PS_ERR_OOM;
  unsigned char* hits = nullptr;
  for (int attempt = 0; attempt < 2; ++attempt) {
    hits = static_cast<unsigned char*>(ws_get(h, WS_HITS, (size_t)cap * 24));
    if (!hits) return PS_ERR_OOM;
    ThreshArgs ta;
    ta.tau = tau;
    ta.bits = bits;
    ta.keys = reinterpret_cast<unsigned long long*>(hits);
    ta.vals = reinterpret_cast<float*>(hits + (size_t)cap * 16);
    ta.counter = counter;
    ta.cap = cap;
    ta.perm = perm;
    PS_CUDA_TRY(h, cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st));
    {
      ScopedTimer tm(h, "threshold3", st);
      PS_CUDA_TRY(h, launch_mgemm3_thresh(h, v, S, n2, dblk, blk.data(), nblocks, ta, st));
    }
    unsigned long long c = 0;
    PS_CUDA_TRY(h, cudaMemcpyAsync(&c, counter, sizeof(c), cudaMemcpyDeviceToHost, st));
    PS_CUDA_TRY(h, cudaStreamSynchronize(st));
    total = (int64_t)c;
    if (total <= cap) break;
    cap = total;  // grow and compute once more
    h->thresh_cap = cap;
  }
  if (total > cap) return fail(h, PS_ERR_CUDA, "threshold hit buffer could not hold %lld hits", (long long)total);
  unsigned long long* keys = reinterpret_cast<unsigned long long*>(hits);
  unsigned long long* ktmp = keys + cap;
  float* vals = reinterpret_cast<float*>(hits + (size_t)cap * 16);
  float* vtmp = vals + cap;
  const size_t words = radix_sort_scratch_words(total);
  unsigned* scratch = static_cast<unsigned*>(ws_get(h, WS_SORT, words * sizeof(unsigned)));
  if (!scratch) return PS_ERR_OOM;
  {
    ScopedTimer tm(h, "sort", st);
    PS_CUDA_TRY(h, launch_radix_sort(h, keys, vals, ktmp, vtmp, total, 3 * bits, scratch, words, st));
  }
  const int64_t nout = std::min(total, capacity);
  OutBuf o;
  if (nout > 0) {
    ps_status s = resolve_out(h, out, (size_t)nout * sizeof(ps_triple), WS_OUTPUT, &o);
    if (s != PS_OK) return s;
    PS_CUDA_TRY(h, launch_write_triples(keys, vals, nout, bits, static_cast<ps_triple*>(o.dev), st));
  }
  OutBuf oc;
  ps_status s2 = resolve_out(h, count, sizeof(int64_t), WS_AUX1, &oc);
  if (s2 != PS_OK) return s2;
  const int64_t tot64 = total;
  PS_CUDA_TRY(h, cudaMemcpyAsync(oc.dev, &tot64, sizeof(int64_t), cudaMemcpyHostToDevice, st));
  if (o.host && o.bytes) PS_CUDA_TRY(h, cudaMemcpyAsync(o.user, o.dev, o.bytes, cudaMemcpyDeviceToHost, st));
  if (oc.host) PS_CUDA_TRY(h, cudaMemcpyAsync(count, oc.dev, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  PS_CUDA_TRY(h, cudaStreamSynchronize(st));
  if (total > capacity)
    return fail(h, PS_ERR_CAPACITY, "%lld triples found, capacity %lld", (long long)total,
                (long long)capacity);
  return PS_OK;
}

}  // namespace
}  // namespace ps

using namespace ps;

extern "C" {

const char* ps_version(void) { return "ps-gb300 0.1 (sm_103a)"; }

const char* ps_status_string(ps_status s) {
  switch (s) {
    case PS_OK: return "PS_OK";
    case PS_ERR_INVALID_ARG: return "PS_ERR_INVALID_ARG";
    case PS_ERR_OOM: return "PS_ERR_OOM";
    case PS_ERR_CUDA: return "PS_ERR_CUDA";
    case PS_ERR_CAPACITY: return "PS_ERR_CAPACITY";
    case PS_ERR_TIMEOUT: return "PS_ERR_TIMEOUT";
    case PS_ERR_UNSUPPORTED: return "PS_ERR_UNSUPPORTED";
  }
  return "PS_ERR_UNKNOWN";
}

const char* ps_last_error(ps_handle h) {
  if (h) return h->last_error.c_str();
  std::lock_guard<std::mutex> g(g_err_mu);
  return g_last_error.c_str();
}

void ps_config_init(ps_config* cfg) {
  if (!cfg) return;
  memset(cfg, 0, sizeof(*cfg));
  cfg->precision = PS_PATH_FP32;
  cfg->wait_limit_ns = 2000000000LL;
}

ps_status ps_create(ps_handle* out, int device, const ps_config* cfg) {
  if (!out) return fail(nullptr, PS_ERR_INVALID_ARG, "ps_create: null out");
  *out = nullptr;
  ps_ctx* h = new (std::nothrow) ps_ctx();
  if (!h) return fail(nullptr, PS_ERR_OOM, "ps_create: out of host memory");
  // the configuration is checked first (host only, no device needed)
  const ps_status cs = apply_config(h, cfg);
  if (cs != PS_OK) {
    const std::string msg = h->last_error;
    delete h;
    return fail(nullptr, cs, "%s", msg.c_str());
  }
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return fail(nullptr, PS_ERR_CUDA, "cudaGetDeviceCount: %s", cudaGetErrorString(e));
  }
  if (device < 0 || device >= n) {
    delete h;
    return fail(nullptr, PS_ERR_INVALID_ARG, "device %d not in [0,%d)", device, n);
  }
  h->device = device;
  Guard g(device);
  cudaDeviceProp prop;
  e = cudaGetDeviceProperties(&prop, device);
  if (e != cudaSuccess) {
    delete h;
    return fail(nullptr, PS_ERR_CUDA, "cudaGetDeviceProperties: %s", cudaGetErrorString(e));
  }
  h->num_sms = prop.multiProcessorCount;
  h->cc_major = prop.major;
  h->cc_minor = prop.minor;
  h->smem_optin = prop.sharedMemPerBlockOptin;
  if (prop.major < 10) {
    delete h;
    return fail(nullptr, PS_ERR_UNSUPPORTED, "device %d is sm_%d%d; this library is built for sm_103a",
                device, prop.major, prop.minor);
  }
  *out = h;
  return PS_OK;
}

ps_status ps_get_config(ps_handle h, ps_config* cfg) {
  if (!h || !cfg) return fail(h, PS_ERR_INVALID_ARG, "ps_get_config: null argument");
  *cfg = h->cfg;
  return PS_OK;
}

ps_status ps_set_config(ps_handle h, const ps_config* cfg) {
  if (!h) return fail(nullptr, PS_ERR_INVALID_ARG, "null handle");
  {
    Guard g(h->device);
    cudaDeviceSynchronize();
  }
  return apply_config(h, cfg);
}

ps_status ps_destroy(ps_handle h) {
  if (!h) return PS_OK;
  {
    Guard g(h->device);
    cudaDeviceSynchronize();
    timing_clear(h);
    if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
    batch_state_free(h);
    mlp_free(h);
    for (int s = 0; s < WS_NUM_SLOTS; ++s)
      if (h->ws.ptr[s]) cudaFree(h->ws.ptr[s]);
    if (h->async_err_host) cudaFreeHost(h->async_err_host);
  }
  delete h;
  return PS_OK;
}

int64_t ps_slab_size(int64_t nv, int64_t j_begin, int64_t j_end) {
  if (nv < 0 || j_begin < 0 || j_end < j_begin || j_end > nv) return -1;
  auto F = [nv](int64_t x) { return (nv - 1) * (x * (x - 1) / 2) - (x - 1) * x * (2 * x - 1) / 6; };
  return F(j_end) - F(j_begin);
}

ps_status ps_vector_sums(ps_handle h, const ps_matrix* V, double* S, ps_stream stream) {
  if (!h) return fail(nullptr, PS_ERR_INVALID_ARG, "null handle");
  ps_status s = check_matrix(h, V, 0);
  if (s != PS_OK) return s;
  if (!S && V->nv > 0) return fail(h, PS_ERR_INVALID_ARG, "null S");
  if (V->nv == 0) return PS_OK;
  Guard g(h->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Prepared P;
  s = prepare(h, *V, st, false, &P);
  if (s != PS_OK) return s;
  OutBuf o;
  s = resolve_out(h, S, (size_t)V->nv * 8, WS_OUTPUT, &o);
  if (s != PS_OK) return s;
  PS_CUDA_TRY(h, cudaMemcpyAsync(o.dev, P.S, (size_t)V->nv * 8, cudaMemcpyDeviceToDevice, st));
  return finish(h, o, P.host_input || o.host, st);
}

ps_status ps_metrics_2way(ps_handle h, const ps_matrix* V, int32_t path, int32_t levels, void* out,
                          int32_t out_dtype, ps_stream stream) {
  if (!h) return fail(nullptr, PS_ERR_INVALID_ARG, "null handle");
  if (const ps_status ae = take_async_error(h); ae != PS_OK) return ae;
  ps_status s = check_matrix(h, V, 2);
  if (s != PS_OK) return s;
  if (!out) return fail(h, PS_ERR_INVALID_ARG, "null out");
  if (out_dtype != PS_F32 && out_dtype != PS_F64 && out_dtype != PS_U8)
    return fail(h, PS_ERR_INVALID_ARG, "out_dtype %d is not PS_F32/PS_F64/PS_U8", out_dtype);
  if (path != PS_PATH_FP32 && path != PS_PATH_FP64 && path != PS_PATH_THERMO && path != PS_PATH_HALF2)
    return fail(h, PS_ERR_INVALID_ARG, "path %d is not a ps_path", path);
  if (out_dtype == PS_U8 && path != PS_PATH_FP32 && path != PS_PATH_THERMO)
    return fail(h, PS_ERR_INVALID_ARG, "PS_U8 output needs PS_PATH_FP32 or PS_PATH_THERMO");
  const bool binary = V->dtype == PS_B1 && path == PS_PATH_THERMO;
  if (path == PS_PATH_THERMO && !binary && (levels < 2 || levels > 16))
    return fail(h, PS_ERR_INVALID_ARG, "levels=%d outside [2,16]", levels);
  Guard g(h->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int64_t npairs = V->nv * (V->nv - 1) / 2;
  const size_t obytes = (size_t)npairs * dtype_size(out_dtype);
  OutBuf o;
  // FP32 path, n_f >= 256 (at most ~8 GB/s of metrics): a pinned or
  // registered host output is written by the kernel itself through its
  // device mapping, with no staging buffer and no copy
  void* direct = (path == PS_PATH_FP32 && V->nf >= 256 && h->host_direct != 1) ? mapped_host(out) : nullptr;
  if (direct) {
    o.dev = direct;
    o.user = out;
    o.host = true;  // (bytes 0: nothing to copy; the call synchronises)
  } else {
    s = resolve_out(h, out, obytes, WS_OUTPUT, &o);
    if (s != PS_OK) return s;
  }
  Prepared P;
  if (binary) {
    s = prepare(h, *V, st, false, &P, false);
    if (s != PS_OK) return s;
    s = binary_2way(h, P.dev, o.dev, out2_mode(out_dtype), st);
    if (s != PS_OK) return s;
  } else if (path == PS_PATH_THERMO) {
    s = prepare(h, *V, st, true, &P, false);
    if (s != PS_OK) return s;
    s = thermo_2way(h, P.f32, levels, o.dev, out2_mode(out_dtype), st);
    if (s != PS_OK) return s;
  } else if (path == PS_PATH_HALF2) {
    s = prepare(h, *V, st, true, &P);
    if (s != PS_OK) return s;
    const int64_t ldh = round_up(V->nv, 4);
    const int64_t np = (V->nf + 1) / 2;
    uint32_t* vh = static_cast<uint32_t*>(ws_get(h, WS_QUANT, (size_t)std::max<int64_t>(np * ldh, 1) * 4));
    unsigned* aux = static_cast<unsigned*>(ws_get(h, WS_AUX3, 256));
    if (!vh || !aux) return PS_ERR_OOM;
    float* inv_scale = reinterpret_cast<float*>(aux + 16);
    {
      ScopedTimer tm(h, "pack", st);
      PS_CUDA_TRY(h, launch_pack_half2(P.f32, vh, ldh, aux, inv_scale, st));
    }
    const VF32 hv{reinterpret_cast<const float*>(vh), ldh, (int)V->nv, (int)np};
    ScopedTimer tm(h, "mgemm2_half", st);
    PS_CUDA_TRY(h, launch_mgemm2_half(h->num_sms, h->mgemm_band, h->mgemm_warps, hv, P.S, o.dev, out_dtype == PS_F64, inv_scale, st));
  } else if (path == PS_PATH_FP32 && o.host && !direct && V->nv >= 8 * 128) {
    // host output: compute in equal-work row bands and copy each finished
    // band (a contiguous packed range) to the host on the handle's copy
    // stream while the next band computes
    s = prepare(h, *V, st, true, &P);
    if (s != PS_OK) return s;
    if (!h->copy_stream) PS_CUDA_TRY(h, cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking));
    constexpr int NB = 8;
    cudaEvent_t ev[NB];
    for (int b = 0; b < NB; ++b) PS_CUDA_TRY(h, cudaEventCreateWithFlags(&ev[b], cudaEventDisableTiming));
    const int keep_tile = h->mgemm_tile;
    h->mgemm_tile = 128;  // bands are whole 128-row tiles
    const size_t esz = dtype_size(out_dtype);
    cudaError_t e = cudaSuccess;
    for (int b = 0; b < NB && e == cudaSuccess; ++b) {
      int64_t rb = 0, re = 0;
      partition_2way(V->nv, NB, b, &rb, &re);
      {
        ScopedTimer tm(h, "mgemm2", st);
        e = launch_mgemm2(h, P.f32, P.S, o.dev, out2_mode(out_dtype), st, (int)(rb / 128),
                          (int)ceil_div(re, 128));
      }
      if (e == cudaSuccess) e = cudaEventRecord(ev[b], st);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(h->copy_stream, ev[b], 0);
      const int64_t ob = rb * (2 * V->nv - rb - 1) / 2, oe = re * (2 * V->nv - re - 1) / 2;
      if (e == cudaSuccess && oe > ob)
        e = cudaMemcpyAsync(static_cast<char*>(o.user) + ob * esz, static_cast<char*>(o.dev) + ob * esz,
                            (size_t)(oe - ob) * esz, cudaMemcpyDeviceToHost, h->copy_stream);
    }
    h->mgemm_tile = keep_tile;
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->copy_stream);
    for (int b = 0; b < NB; ++b) cudaEventDestroy(ev[b]);
    PS_CUDA_TRY(h, e);
    o.bytes = 0;  // already copied
  } else if (path == PS_PATH_FP32) {
    s = prepare(h, *V, st, true, &P);
    if (s != PS_OK) return s;
    ScopedTimer tm(h, "mgemm2", st);
    PS_CUDA_TRY(h, launch_mgemm2(h, P.f32, P.S, o.dev, out2_mode(out_dtype), st));
  } else {  // PS_PATH_FP64: FP64 field-major operand
    s = prepare(h, *V, st, false, &P);
    if (s != PS_OK) return s;
    const double* X;
    int64_t ld;
    s = fp64_operand(h, V, P, st, &X, &ld);
    if (s != PS_OK) return s;
    ScopedTimer tm(h, "mgemm2_f64", st);
    PS_CUDA_TRY(h, launch_mgemm2_f64(h, X, ld, (int)V->nv, (int)V->nf, P.S, o.dev,
                                     out_dtype == PS_F64, st));
  }
  return finish(h, o, P.host_input || o.host, st);
}

ps_status ps_partition(int64_t nv, int32_t way, int32_t nparts, int32_t part, int64_t* begin,
                       int64_t* end, int64_t* out_begin, int64_t* out_end) {
  if (nv < way || (way != 2 && way != 3) || nparts < 1 || part < 0 || part >= nparts || !begin || !end)
    return fail(nullptr, PS_ERR_INVALID_ARG, "ps_partition: bad arguments");
  if (way == 2) {
    partition_2way(nv, nparts, part, begin, end);
    auto idx = [nv](int64_t i) { return i * (2 * nv - i - 1) / 2; };  // first pair of row i
    if (out_begin) *out_begin = idx(*begin);
    if (out_end) *out_end = idx(*end);
  } else {
    partition_3way(nv, nparts, part, begin, end);
    if (out_begin) *out_begin = ps_slab_size(nv, 0, *begin);
    if (out_end) *out_end = ps_slab_size(nv, 0, *end);
  }
  return PS_OK;
}

ps_status ps_metrics_2way_part(ps_handle h, const ps_matrix* V, int32_t nparts, int32_t part,
                               void* out, int32_t out_dtype, ps_stream stream) {
  if (!h) return fail(nullptr, PS_ERR_INVALID_ARG, "null handle");
  if (const ps_status ae = take_async_error(h); ae != PS_OK) return ae;
  ps_status s = check_matrix(h, V, 2);
  if (s != PS_OK) return s;
  if (nparts < 1 || part < 0 || part >= nparts) return fail(h, PS_ERR_INVALID_ARG, "part %d of %d", part, nparts);
  if (!out) return fail(h, PS_ERR_INVALID_ARG, "null out");
  if (out_dtype != PS_F32 && out_dtype != PS_F64 && out_dtype != PS_U8)
    return fail(h, PS_ERR_INVALID_ARG, "out_dtype %d is not PS_F32/PS_F64/PS_U8", out_dtype);
  Guard g(h->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int64_t rb = 0, re = 0;
  partition_2way(V->nv, nparts, part, &rb, &re);
  const int64_t npairs = V->nv * (V->nv - 1) / 2;
  OutBuf o;
  s = resolve_out(h, out, (size_t)npairs * dtype_size(out_dtype), WS_OUTPUT, &o);
  if (s != PS_OK) return s;
  if (o.host) return fail(h, PS_ERR_INVALID_ARG, "ps_metrics_2way_part needs a device output");
  if (wants_fp64(h)) {
    // the paper's DP arithmetic: the FP64 kernel over the same rows
    if (out_dtype == PS_U8) return fail(h, PS_ERR_UNSUPPORTED, "PS_U8 output under FP64 precision");
    Prepared P;
    s = prepare(h, *V, st, false, &P);
    if (s != PS_OK) return s;
    const double* X;
    int64_t ld;
    s = fp64_operand(h, V, P, st, &X, &ld);
    if (s != PS_OK) return s;
    ScopedTimer tm(h, "mgemm2_f64", st);
    PS_CUDA_TRY(h, launch_mgemm2_f64(h, X, ld, (int)V->nv, (int)V->nf, P.S, o.dev, out_dtype == PS_F64, st, rb,
                                     re));
    return finish(h, o, P.host_input, st);
  }
  Prepared P;
  s = prepare(h, *V, st, true, &P);
  if (s != PS_OK) return s;
  {
    ScopedTimer tm(h, "mgemm2", st);
    // row bands are whole 128-row tiles; the kernels use 128-wide tiles here
    const int keep_tile = h->mgemm_tile;
    h->mgemm_tile = 128;  // (8 or 16 warps per 128 x 128 tile as configured)
    const cudaError_t e = launch_mgemm2(h, P.f32, P.S, o.dev, out2_mode(out_dtype), st, (int)(rb / 128),
                                        (int)ceil_div(re, 128));
    h->mgemm_tile = keep_tile;
    PS_CUDA_TRY(h, e);
  }
  return finish(h, o, P.host_input, st);
}

ps_status ps_metrics_3way(ps_handle h, const ps_matrix* V, int64_t j_begin, int64_t j_end,
                          float* out_slab, ps_stream stream) {
  if (!h) return fail(nullptr, PS_ERR_INVALID_ARG, "null handle");
  if (const ps_status ae = take_async_error(h); ae != PS_OK) return ae;
  ps_status s = check_matrix(h, V, 3);
  if (s != PS_OK) return s;
  if (wants_fp64(h))
    return fail(h, PS_ERR_UNSUPPORTED, "%s has no FP64 kernel (handle precision is PS_PATH_FP64)", "ps_metrics_3way");
  if (j_begin < 0 || j_end < j_begin || j_end > V->nv)
    return fail(h, PS_ERR_INVALID_ARG, "pivot range [%lld,%lld) not inside [0,%lld]",
                (long long)j_begin, (long long)j_end, (long long)V->nv);
  const int64_t n = ps_slab_size(V->nv, j_begin, j_end);
  if (n > 0 && !out_slab) return fail(h, PS_ERR_INVALID_ARG, "null out_slab");
  if (n == 0) return PS_OK;
  Guard g(h->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  OutBuf o;
  s = resolve_out(h, out_slab, (size_t)n * 4, WS_OUTPUT, &o);
  if (s != PS_OK) return s;
  Prepared P;
  s = prepare(h, *V, st, true, &P);
  if (s != PS_OK) return s;
  float* n2 = static_cast<float*>(ws_get(h, WS_N2, (size_t)V->nv * V->nv * 4));
  if (!n2) return PS_ERR_OOM;
  {
    ScopedTimer tm(h, "mgemm2_n2", st);
    PS_CUDA_TRY(h, launch_mgemm2(h, P.f32, P.S, n2, OUT2_N2_SQUARE_F32, st));
  }
  {
    ScopedTimer tm(h, "mgemm3", st);
    PS_CUDA_TRY(h, launch_mgemm3(h, P.f32, P.S, n2, j_begin, j_end, static_cast<float*>(o.dev), st));
  }
  return finish(h, o, P.host_input || o.host, st);
}

ps_status ps_threshold_3way(ps_handle h, const ps_matrix* V, float tau, int32_t use_proposal,
                            ps_triple* out, int64_t capacity, int64_t* count, ps_stream stream) {
  if (!h) return fail(nullptr, PS_ERR_INVALID_ARG, "null handle");
  if (const ps_status ae = take_async_error(h); ae != PS_OK) return ae;
  ps_status s = check_matrix(h, V, 3);
  if (s != PS_OK) return s;
  if (wants_fp64(h))
    return fail(h, PS_ERR_UNSUPPORTED, "%s has no FP64 kernel (handle precision is PS_PATH_FP64)", "ps_threshold_3way");
  if (V->nv > (1 << 21)) return fail(h, PS_ERR_INVALID_ARG, "nv=%lld above 2^21", (long long)V->nv);
  if (capacity < 0) return fail(h, PS_ERR_INVALID_ARG, "capacity < 0");
  if (!count) return fail(h, PS_ERR_INVALID_ARG, "null count");
  if (capacity > 0 && !out) return fail(h, PS_ERR_INVALID_ARG, "null out");
  if (use_proposal < 0 || use_proposal > 2)
    return fail(h, PS_ERR_INVALID_ARG, "use_proposal %d is not 0, 1 or 2", use_proposal);
  if (use_proposal == 1 && !h->mlp.trained)
    return fail(h, PS_ERR_INVALID_ARG, "use_proposal 1 needs a trained encoder (ps_proposal_train)");
  if (use_proposal == 1 && V->nf != h->mlp.d_in)
    return fail(h, PS_ERR_INVALID_ARG, "encoder expects nf=%d", h->mlp.d_in);
  Guard g(h->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Prepared P;
  s = prepare(h, *V, st, true, &P);
  if (s != PS_OK) return s;
  const int nv = (int)V->nv;
  // reorder by the encoder's clusters when a proposal is asked for and an
  // encoder is trained for this n_f
  VF32 v = P.f32;
  double* S = P.S;
  int* perm = nullptr;
  if (use_proposal != 0 && h->mlp.trained && V->nf == h->mlp.d_in) {
    s = proposal_reorder(h, P.f32, P.S, st, &v, &S, &perm);
    if (s != PS_OK) return s;
  }
  float* n2 = static_cast<float*>(ws_get(h, WS_N2, (size_t)nv * nv * 4));
  if (!n2) return PS_ERR_OOM;
  {
    ScopedTimer tm(h, "mgemm2_n2", st);
    PS_CUDA_TRY(h, launch_mgemm2(h, v, S, n2, OUT2_N2_SQUARE_F32, st));
  }
  std::vector<int> blk;
  double kept = 1.0;
  if (use_proposal == 1) {
    s = proposal_blocks_learned(h, v, S, st, &blk, &kept);
    if (s != PS_OK) return s;
  } else if (use_proposal == 2) {
    s = proposal_blocks_bound(h, v, S, n2, tau, st, &blk, &kept);
    if (s != PS_OK) return s;
  }
  if (use_proposal == 0 || (use_proposal == 1 && kept > 0.6)) {
    // exhaustive: every block (I <= Jt <= K) of 128-wide tiles (also the
    // fallback when the learned proposal would keep most blocks anyway)
    const int T = (int)ceil_div(nv, 128);
    blk.clear();
    for (int I = 0; I < T; ++I)
      for (int K = I; K < T; ++K)
        for (int Jt = I; Jt <= K; ++Jt) {
          blk.push_back(I);
          blk.push_back(Jt);
          blk.push_back(K);
        }
    kept = 1.0;
  }
  h->last_kept = kept;
  h->last_blocks = (int64_t)blk.size() / 3;
  return threshold_blocks(h, v, S, perm, blk, tau, out, capacity, count, st);
}

ps_status ps_threshold_2way(ps_handle h, const ps_matrix* V, float tau, ps_pair* out, int64_t capacity,
                            int64_t* count, ps_stream stream) {
  if (!h) return fail(nullptr, PS_ERR_INVALID_ARG, "null handle");
  ps_status s = check_matrix(h, V, 2);
  if (s != PS_OK) return s;
  if (wants_fp64(h))
    return fail(h, PS_ERR_UNSUPPORTED, "%s has no FP64 kernel (handle precision is PS_PATH_FP64)", "ps_threshold_2way");
  if (V->nv > 2147483647LL) return fail(h, PS_ERR_INVALID_ARG, "nv=%lld above 2^31-1", (long long)V->nv);
  if (capacity < 0) return fail(h, PS_ERR_INVALID_ARG, "capacity < 0");
  if (!count) return fail(h, PS_ERR_INVALID_ARG, "null count");
  if (capacity > 0 && !out) return fail(h, PS_ERR_INVALID_ARG, "null out");
  Guard g(h->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Prepared P;
  s = prepare(h, *V, st, true, &P);
  if (s != PS_OK) return s;
  const int bits = key_bits_for((int)V->nv);
  int64_t cap = std::max<int64_t>({capacity, (int64_t)1 << 20, h->thresh_cap});
  unsigned long long* counter = static_cast<unsigned long long*>(ws_get(h, WS_AUX3, 256));
  if (!counter) return PS_ERR_OOM;
  int64_t total = 0;
  unsigned char* hits = nullptr;
  for (int attempt = 0; attempt < 2; ++attempt) {
    hits = static_cast<unsigned char*>(ws_get(h, WS_HITS, (size_t)cap * 24));
    if (!hits) return PS_ERR_OOM;
    ThreshArgs ta;
    ta.tau = tau;
    ta.bits = bits;
    ta.keys = reinterpret_cast<unsigned long long*>(hits);
    ta.vals = reinterpret_cast<float*>(hits + (size_t)cap * 16);
    ta.counter = counter;
    ta.cap = cap;
    ta.perm = nullptr;
    PS_CUDA_TRY(h, cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st));
    {
      ScopedTimer tm(h, "threshold2", st);
      if (h->mgemm_feed_tma && V->nf > 0) {
        // the TMA-fed pipeline (default); mgemm_feed = 2: the cp.async kernel
        int* err = async_err_word(h);
        if (!err) return PS_ERR_OOM;
        PS_CUDA_TRY(h, launch_mgemm2_thresh_tma(h, P.f32, P.S, ta, st, err));
      } else {
        PS_CUDA_TRY(h, launch_mgemm2_thresh(h->num_sms, h->mgemm_band, P.f32, P.S, ta, st));
      }
    }
    unsigned long long c = 0;
    PS_CUDA_TRY(h, cudaMemcpyAsync(&c, counter, sizeof(c), cudaMemcpyDeviceToHost, st));
    PS_CUDA_TRY(h, cudaStreamSynchronize(st));
    total = (int64_t)c;
    if (total <= cap) break;
    cap = total;  // grow and compute once more
    h->thresh_cap = cap;
  }
  if (total > cap) return fail(h, PS_ERR_CUDA, "threshold hit buffer could not hold %lld hits", (long long)total);
  unsigned long long* keys = reinterpret_cast<unsigned long long*>(hits);
  float* vals = reinterpret_cast<float*>(hits + (size_t)cap * 16);
  const size_t words = radix_sort_scratch_words(total);
  unsigned* scratch = static_cast<unsigned*>(ws_get(h, WS_SORT, words * sizeof(unsigned)));
  if (!scratch) return PS_ERR_OOM;
  {
    ScopedTimer tm(h, "sort", st);
    PS_CUDA_TRY(h, launch_radix_sort(h, keys, vals, keys + cap, vals + cap, total, 2 * bits, scratch, words, st));
  }
  const int64_t nout = std::min(total, capacity);
  OutBuf o;
  if (nout > 0) {
    s = resolve_out(h, out, (size_t)nout * sizeof(ps_pair), WS_OUTPUT, &o);
    if (s != PS_OK) return s;
    PS_CUDA_TRY(h, launch_write_pairs(keys, vals, nout, bits, static_cast<ps_pair*>(o.dev), st));
  }
  OutBuf oc;
  s = resolve_out(h, count, sizeof(int64_t), WS_AUX1, &oc);
  if (s != PS_OK) return s;
  const int64_t tot64 = total;
  PS_CUDA_TRY(h, cudaMemcpyAsync(oc.dev, &tot64, sizeof(int64_t), cudaMemcpyHostToDevice, st));
  if (o.host && o.bytes) PS_CUDA_TRY(h, cudaMemcpyAsync(o.user, o.dev, o.bytes, cudaMemcpyDeviceToHost, st));
  if (oc.host) PS_CUDA_TRY(h, cudaMemcpyAsync(count, oc.dev, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  PS_CUDA_TRY(h, cudaStreamSynchronize(st));
  if (total > capacity)
    return fail(h, PS_ERR_CAPACITY, "%lld pairs found, capacity %lld", (long long)total, (long long)capacity);
  return PS_OK;
}

ps_status ps_proposal_last_stats(ps_handle h, double* kept_fraction, int64_t* blocks) {
  if (!h || !kept_fraction || !blocks) return fail(h, PS_ERR_INVALID_ARG, "null argument");
  *kept_fraction = h->last_kept;
  *blocks = h->last_blocks;
  return PS_OK;
}

ps_status ps_quantize(ps_handle h, const ps_matrix* V, int32_t levels, float* P_out, uint8_t* q_out,
                      ps_stream stream) {
  if (!h) return fail(nullptr, PS_ERR_INVALID_ARG, "null handle");
  ps_status s = check_matrix(h, V, 1);
  if (s != PS_OK) return s;
  if (levels < 2 || levels > 16) return fail(h, PS_ERR_INVALID_ARG, "levels=%d outside [2,16]", levels);
  if (!P_out) return fail(h, PS_ERR_INVALID_ARG, "null P_out");
  Guard g(h->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Prepared P;
  s = prepare(h, *V, st, true, &P, false);
  if (s != PS_OK) return s;
  SelectState* sel = nullptr;
  s = run_percentile(h, P.f32, st, &sel);
  if (s != PS_OK) return s;
  OutBuf oP;
  s = resolve_out(h, P_out, sizeof(float), WS_AUX3, &oP);
  if (s != PS_OK) return s;
  PS_CUDA_TRY(h, cudaMemcpyAsync(oP.dev, &sel->value, sizeof(float), cudaMemcpyDeviceToDevice, st));
  OutBuf oq;
  if (q_out) {
    s = resolve_out(h, q_out, (size_t)V->nv * V->nf, WS_OUTPUT, &oq);
    if (s != PS_OK) return s;
    PS_CUDA_TRY(h, launch_quantize(P.f32, levels, sel, static_cast<uint8_t*>(oq.dev), V->nv, st));
  }
  if (oP.host) PS_CUDA_TRY(h, cudaMemcpyAsync(P_out, oP.dev, sizeof(float), cudaMemcpyDeviceToHost, st));
  return finish(h, oq, P.host_input || oP.host || oq.host, st);
}

ps_status ps_timing_enable(ps_handle h, int32_t enable) {
  if (!h) return fail(nullptr, PS_ERR_INVALID_ARG, "null handle");
  Guard g(h->device);
  timing_clear(h);
  h->timing = enable != 0;
  return PS_OK;
}

ps_status ps_timing_read(ps_handle h, const char* kernel, int64_t* launches, double* total_ms) {
  if (!h || !kernel || !launches || !total_ms)
    return fail(h, PS_ERR_INVALID_ARG, "ps_timing_read: null argument");
  Guard g(h->device);
  int64_t n = 0;
  double ms = 0.0;
  for (auto& r : h->trecs) {
    if (strcmp(r.name, kernel) != 0) continue;
    PS_CUDA_TRY(h, cudaEventSynchronize(r.b));
    float t = 0.f;
    PS_CUDA_TRY(h, cudaEventElapsedTime(&t, r.a, r.b));
    ms += t;
    ++n;
  }
  *launches = n;
  *total_ms = ms;
  return PS_OK;
}

ps_status ps_probe_minadd_peak(ps_handle h, int32_t variant, double* cmp_per_s) {
  if (!h) return fail(nullptr, PS_ERR_INVALID_ARG, "null handle");
  if (variant < 0 || variant > 4) return fail(h, PS_ERR_INVALID_ARG, "variant %d", variant);
  if (!cmp_per_s) return fail(h, PS_ERR_INVALID_ARG, "null cmp_per_s");
  Guard g(h->device);
  PS_CUDA_TRY(h, probe_minadd(h, variant, cmp_per_s));
  return PS_OK;
}

}  // extern "C"
