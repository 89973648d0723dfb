// Exhaustive device check of ps::div_rn_lean against __fdiv_rn.
//
// 1. rcp.approx(d 2^E) == rcp.approx(d) 2^-E for every significand of d and
//    every E in [-81, 101] (the division's range of denominators), so the
//    reciprocal step scales exactly with the exponent of d.
// 2. div_rn_lean(x, d) == __fdiv_rn(x, d), bit for bit, for every pair of
//    significands x, d in [1, 2) (2^46 pairs) and for x = 0.
// Prints one line "mismatches R Q Z" (reciprocal, quotient, zero cases) and
// exits 0 when the run itself succeeded; the caller checks the counts.
#include <cstdint>
#include <cstdio>

#include "../paper_1705_08210_gb300/csrc/ps_div.cuh"

namespace {

constexpr uint32_t NSIG = 1u << 23;   // significands of [1, 2)
constexpr uint32_t XCH = 1024;        // x ranges per d
constexpr uint32_t XPER = NSIG / XCH; // x significands per thread

__device__ __forceinline__ float rcp_approx(float d) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(d));
  return y;
}

__global__ void rcp_scale(unsigned long long* bad) {
  const uint32_t m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= NSIG) return;
  const uint32_t y0 = __float_as_uint(rcp_approx(__uint_as_float(0x3f800000u | m)));
  unsigned b = 0;
  for (int E = -81; E <= 101; ++E) {
    const float d = __uint_as_float(((uint32_t)(127 + E) << 23) | m);
    // y0 is normal in (0.5, 1]: scaling by 2^-E subtracts E from its exponent field
    if (__float_as_uint(rcp_approx(d)) != y0 - ((uint32_t)E << 23)) ++b;
  }
  if (b) atomicAdd(bad, (unsigned long long)b);
}

// threads g = (d index - d0) * XCH + x range; each covers XPER values of x
__global__ void quotients(uint32_t d0, uint32_t nd, unsigned long long* bad) {
  const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= (uint64_t)nd * XCH) return;
  const uint32_t di = d0 + (uint32_t)(g / XCH);
  const uint32_t x0 = (uint32_t)(g % XCH) * XPER;
  const float d = __uint_as_float(0x3f800000u | di);
  unsigned b = 0;
  for (uint32_t m = x0; m < x0 + XPER; ++m) {
    const float x = __uint_as_float(0x3f800000u | m);
    if (__float_as_uint(ps::div_rn_lean(x, d)) != __float_as_uint(__fdiv_rn(x, d))) ++b;
  }
  if (b) atomicAdd(bad, (unsigned long long)b);
}

__global__ void zeros(unsigned long long* bad) {
  const uint32_t m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= NSIG) return;
  for (int E = -81; E <= 101; E += 13) {
    const float d = __uint_as_float(((uint32_t)(127 + E) << 23) | m);
    if (__float_as_uint(ps::div_rn_lean(0.0f, d)) != 0u) atomicAdd(bad, 1ull);
  }
}

bool ok(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return true;
  std::printf("error %s: %s\n", what, cudaGetErrorString(e));
  return false;
}

}  // namespace

int main() {
  unsigned long long* bad = nullptr;
  if (!ok(cudaMalloc(&bad, 3 * sizeof(unsigned long long)), "alloc")) return 1;
  if (!ok(cudaMemset(bad, 0, 3 * sizeof(unsigned long long)), "memset")) return 1;
  rcp_scale<<<NSIG / 256, 256>>>(bad);
  zeros<<<NSIG / 256, 256>>>(bad + 2);
  if (!ok(cudaDeviceSynchronize(), "reciprocal sweep")) return 1;
  // 64 launches of 131072 denominators each, about a second apiece
  constexpr uint32_t ND = NSIG / 64;
  for (uint32_t d0 = 0; d0 < NSIG; d0 += ND) {
    const uint64_t threads = (uint64_t)ND * XCH;
    quotients<<<(unsigned)(threads / 256), 256>>>(d0, ND, bad + 1);
    if (!ok(cudaDeviceSynchronize(), "quotient sweep")) return 1;
  }
  unsigned long long h[3];
  if (!ok(cudaMemcpy(h, bad, sizeof h, cudaMemcpyDeviceToHost), "copy")) return 1;
  std::printf("mismatches %llu %llu %llu\n", h[0], h[1], h[2]);
  cudaFree(bad);
  return 0;
}
