// ps_static.cu -- 2-way metrics without any device allocation.
//
// ps_metrics_2way needs scratch device memory for the FP64 per-vector sums
// (and, for inputs the kernel cannot read directly, a repacked FP32 copy),
// which it takes from a workspace grown with cudaMalloc.  Some callers cannot
// let a library call cudaMalloc: services whose device memory is owned in full
// by their own allocator or a fixed budget set at start-up (a framework's
// caching allocator that must account for every byte, a long-running service
// that forbids cudaMalloc/cudaFree after warm-up because they can synchronise
// the device and fragment memory).  ps_metrics_2way_static serves them: the
// only scratch it uses is the file-scope array below, so the call itself
// allocates nothing.
//
// The array is part of the library's device image: every GPU on which the
// library's kernels are loaded holds it (512 KiB) until the process exits.
// All calls share it and it keeps the last call's contents; each call
// rewrites the sums of its own vectors before reading them, so nothing has to
// start at zero.  Calls that overlap on the GPU (different streams, or
// different host threads) race on the array: serialise them.
#include "ps_internal.cuh"

namespace ps {
namespace {

constexpr int64_t kStaticMaxNv = 65536;  // = PS_STATIC_MAX_NV in ps.h

// Scratch of the no-allocation entry point: per-vector FP64 sums.
static __device__ __align__(256) double g_static_sums[kStaticMaxNv];

// Device address of g_static_sums on the current device.  In host code the
// name g_static_sums is only a host-side stand-in, so the kernels get the
// address cudaGetSymbolAddress returns.  It is looked up on every call (a
// host-side query that allocates nothing), so a context that was torn down
// and created again, which may load the module at another address, never
// receives a stale pointer.  The first lookup on a device loads the module
// there; make that first call before any stream capture.
cudaError_t static_sums_address(double** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_static_sums);
  if (e != cudaSuccess) return e;
  *out = static_cast<double*>(p);
  return cudaSuccess;
}

bool is_device_pointer(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace ps

using namespace ps;

extern "C" ps_status ps_metrics_2way_static(const ps_matrix* V, void* out, int32_t out_dtype,
                                            ps_stream stream) {
  if (!V) return fail(nullptr, PS_ERR_INVALID_ARG, "ps_metrics_2way_static: null matrix");
  if (V->nv < 2 || V->nv > kStaticMaxNv)
    return fail(nullptr, PS_ERR_INVALID_ARG,
                "ps_metrics_2way_static: nv=%lld outside [2, %lld] (the size of the static scratch)",
                (long long)V->nv, (long long)kStaticMaxNv);
  if (V->nf < 0 || V->nf > ((int64_t)1 << 30))
    return fail(nullptr, PS_ERR_INVALID_ARG, "ps_metrics_2way_static: nf=%lld", (long long)V->nf);
  if (V->dtype != PS_F32 || V->layout != PS_LAYOUT_FIELD_MAJOR)
    return fail(nullptr, PS_ERR_INVALID_ARG,
                "ps_metrics_2way_static: needs PS_F32 PS_LAYOUT_FIELD_MAJOR input (no repacking)");
  if (V->ld < V->nv || V->ld % 4 != 0)
    return fail(nullptr, PS_ERR_INVALID_ARG,
                "ps_metrics_2way_static: ld=%lld must be >= nv and a multiple of 4", (long long)V->ld);
  if (!out || (V->nf > 0 && !V->data))
    return fail(nullptr, PS_ERR_INVALID_ARG, "ps_metrics_2way_static: null pointer");
  if (V->nf > 0 && ((uintptr_t)V->data % 16) != 0)
    return fail(nullptr, PS_ERR_INVALID_ARG, "ps_metrics_2way_static: data not 16-byte aligned");
  if (out_dtype != PS_F32 && out_dtype != PS_F64)
    return fail(nullptr, PS_ERR_INVALID_ARG, "ps_metrics_2way_static: out_dtype %d", out_dtype);
  if ((V->nf > 0 && !is_device_pointer(V->data)) || !is_device_pointer(out))
    return fail(nullptr, PS_ERR_INVALID_ARG,
                "ps_metrics_2way_static: data and out must be device memory (no host staging)");

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetDevice");
  double* S = nullptr;
  e = static_sums_address(&S);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetSymbolAddress(g_static_sums)");
  // stack context with the default configuration: no workspace is touched by
  // the calls below; the 16-warp 128 x 128 cp.async kernel (it needs no
  // error word) gives the same values as the default TMA-fed kernel
  ps_ctx ctx;
  ctx.device = dev;
  ctx.mgemm_feed_tma = 0;
  e = cudaDeviceGetAttribute(&ctx.num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaDeviceGetAttribute");

  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  e = launch_vector_sums(*V, S, st);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "vector sums");
  const VF32 v32{static_cast<const float*>(V->data), V->ld, (int)V->nv, (int)V->nf};
  e = launch_mgemm2(&ctx, v32, S, out, out_dtype == PS_F64 ? OUT2_C2_F64 : OUT2_C2_F32, st);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "min-product kernel");
  return PS_OK;
}
