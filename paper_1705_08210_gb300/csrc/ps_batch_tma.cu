// ps_batch_tma.cu -- the persistent batched launch on the TMA-fed pipeline.
//
// Not in the paper (its unit of work is one large decomposed problem, §4).
// One persistent kernel over a work list that mixes the tiles of many
// independent problems: 2-way tiles (Section 2.1's c2 over the upper
// triangle, Section 3.1), n2-table tiles of the 3-way problems, and 3-way
// work items (pivot j, row tile I, column tile K; Section 3.2's B_j = X_j^T
// (min) V restricted to i < j < k).  The per-vector sums come from a
// separate launch before it (batched_sums_kernel), so no tile waits for
// them.
//
// Pipeline (as the TMA-fed 2-way and 3-way kernels): 16 warps, a 3-stage
// shared-memory ring of 64-field slices guarded by full / ready / empty
// mbarriers; lane 0 of warp 0 is the producer.  It claims the next work
// item from a grid-wide counter (one item ahead of its use), reads the
// item's problem record (whose tensor maps live in global memory, 128-byte
// aligned, written before the launch), and issues per slice two 2-D TMA
// loads (row panel, column panel) plus, for a 3-way item, a 4-vector box
// holding the pivot column.  Items have different n_f, so each item
// contributes its own number of slices; the producer hands the item index
// to the warps through tile_of and, per stage, the pivot's column in the box
// (or -1: no pivot).  One slice ahead of the compute each warp applies the
// pivot min to its rows of the row panel (nothing for 2-way items) and
// arrives on the stage's `ready` barrier.
//
// Dependencies: a 3-way item's epilogue reads its problem's n2 table, which
// the same launch writes in n2 tiles that precede every 3-way item in the
// work list.  Each warp counts its finished n2-tile stores on the problem's
// counter (after a memory fence); a 3-way epilogue waits (bounded, lane 0
// polls with acquire loads) until the counter reaches 16 x the problem's n2
// tiles.  Every awaited store belongs to an item claimed earlier, by a CTA
// that waits on nothing later (n2 tiles wait on nothing), so the waits end.
//
// Values: the same micro-kernel, fold schedule (every 64 fields) and
// epilogues as the single-problem kernels, so every output equals
// ps_metrics_2way / ps_metrics_3way's bit for bit.
#include "ps_mgemm_impl.cuh"
#include "ps_sync.cuh"

#include <algorithm>
#include <mutex>

namespace ps {
namespace {

using C = mg::T128W16;
constexpr int NW = C::NT / 32;
// 64-field slices in a 3-slice ring (as the single-problem 3-way kernel,
// which carries most of a batch's comparisons: the pivot min, waits and
// releases per field halve against 32-field slices)
constexpr int BKB = 64;      // fields per slice
constexpr int STAGES_B = 3;  // ring depth
constexpr int PBOX = 4;      // pivot box: 4 vectors x BKB fields

struct __align__(128) SmemB {
  float A[STAGES_B][BKB][C::BM];
  float B[STAGES_B][BKB][C::BN];
  float P[STAGES_B][BKB][PBOX];
  int pcol[STAGES_B];     // pivot column in the box, -1: no pivot (2-way or n2 item)
  int tile_of[STAGES_B];  // work item of local item lt at [lt % STAGES_B], -1: none left
  unsigned long long full[STAGES_B];
  unsigned long long ready[STAGES_B];
  unsigned long long empty[STAGES_B];
  // producer state (thread 0): current item, its slice, its slice count
  int p_item, p_kb, p_nkb, p_done;
  int abort;
};

__device__ __forceinline__ int ld_acquire_s32(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Lane 0 waits until *ctr >= target (bounded), the warp follows its verdict.
__device__ __forceinline__ bool warp_wait_count(const int* ctr, int target, int* abort_word, int* err,
                                                unsigned long long wait_ns) {
  int ok = 1;
  if ((threadIdx.x & 31) == 0 && ld_acquire_s32(ctr) < target) {
    const unsigned long long t0 = sy::now_ns();
    for (;;) {
      __nanosleep(128);
      if (ld_acquire_s32(ctr) >= target) break;
      if (*(volatile int*)abort_word || *(volatile int*)err) {
        *(volatile int*)abort_word = 1;  // the CTA's other warps stop waiting too
        ok = 0;
        break;
      }
      if (sy::now_ns() - t0 > wait_ns) {
        *(volatile int*)abort_word = 1;
        atomicExch(err, 1);
        __threadfence_system();
        ok = 0;
        break;
      }
    }
  }
  return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

__global__ void __launch_bounds__(C::NT, 1)
    batched_tma_kernel(const BatchProbTma* __restrict__ probs, const BatchItem* __restrict__ items, int nitems,
                       int* __restrict__ counters, unsigned long long wait_ns) {
  constexpr int FOLD_SLICES = mg::FOLD * mg::BK / BKB;  // 64 fields per compensated fold
  constexpr int ROWS_PER_WARP = BKB / NW;
  constexpr uint32_t PANELS = 2u * BKB * C::BM * sizeof(float);
  constexpr uint32_t PIVOT = BKB * PBOX * sizeof(float);
  extern __shared__ __align__(128) unsigned char smem_raw[];
  SmemB& sm = *reinterpret_cast<SmemB*>(smem_raw);
  int* queue = counters;
  int* err = counters + 1;
  int* n2_done = counters + 2;  // per problem: n2-tile warp stores finished
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES_B; ++s) {
      sy::bar_init(&sm.full[s], 1);
      sy::bar_init(&sm.ready[s], NW);
      sy::bar_init(&sm.empty[s], NW);
    }
    sm.abort = 0;
    sm.p_kb = 0;
    sm.p_nkb = 0;
    sm.p_done = 0;
    sy::bar_init_fence();
  }
  __syncthreads();
  const bool producer = threadIdx.x == 0;
  int next_claim = 0;
  if (producer) next_claim = atomicAdd(queue, 1);
  uint32_t p_g = 0;  // producer: next slice of this CTA's sequence
  int p_r = 0;       // producer: local index of the current item

  // producer: issues the next slice of this CTA's sequence (waiting until
  // its stage is free); false on abort
  auto issue_one = [&]() -> bool {
    SmemB& sm = *reinterpret_cast<SmemB*>(smem_raw);
    if (sm.p_done) return true;
    const int s = (int)(p_g % STAGES_B);
    const uint32_t ph = (p_g / STAGES_B) & 1u;
    if (!sy::bar_wait(&sm.empty[s], ph ^ 1u, &sm.abort, err, wait_ns)) return false;
    if (sm.p_kb == 0) {
      // (the stage being free means every warp has read entry p_r - STAGES_B)
      const int t = next_claim;
      if (t < nitems) next_claim = atomicAdd(queue, 1);
      if (t >= nitems) {
        sm.tile_of[p_r % STAGES_B] = -1;
        sy::bar_arrive(&sm.full[s]);  // completes the phase with no copies: the warps stop
        sm.p_done = 1;
        return true;
      }
      sm.tile_of[p_r % STAGES_B] = t;  // published by the arrival below
      sm.p_item = t;
      const BatchProbTma* pt = probs + __ldg(&items[t].prob);
      sm.p_nkb = max(1, (__ldg(&pt->nf) + BKB - 1) / BKB);
      // the maps were written through the generic proxy (before the launch)
      asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&pt->mapV) : "memory");
      asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&pt->mapP) : "memory");
    }
    const BatchItem w = items[sm.p_item];
    const BatchProbTma* pr = probs + w.prob;
    int row0, col0, pj = -1;
    if (w.kind == BK_TILE3) {
      pj = w.a;
      row0 = (w.b >> 16) * C::BM;
      col0 = (w.b & 0xffff) * C::BN;
    } else {
      row0 = w.a * C::BM;
      col0 = w.b * C::BN;
    }
    const int kb = sm.p_kb;
    sm.pcol[s] = pj < 0 ? -1 : (pj & (PBOX - 1));
    sy::bar_arrive_tx(&sm.full[s], pj < 0 ? PANELS : PANELS + PIVOT);
    sy::tma_load_2d(&sm.A[s][0][0], &pr->mapV, row0, kb * BKB, &sm.full[s]);
    sy::tma_load_2d(&sm.B[s][0][0], &pr->mapV, col0, kb * BKB, &sm.full[s]);
    if (pj >= 0) sy::tma_load_2d(&sm.P[s][0][0], &pr->mapP, pj & ~(PBOX - 1), kb * BKB, &sm.full[s]);
    ++p_g;
    if (++sm.p_kb == sm.p_nkb) {
      sm.p_kb = 0;
      ++p_r;
    }
    return true;
  };
  if (producer)
    for (int p = 0; p + 1 < STAGES_B; ++p)
      if (!issue_one()) break;

  // slice g: wait for its copies, apply the pivot min to this warp's rows
  // (3-way items), arrive on `ready`.  first_of_item: g starts an item, whose
  // entry may be the end marker (then there is nothing to prepare).
  auto prepare = [&](uint32_t g, int lt_of_g, bool first_of_item) -> bool {
    SmemB& sm = *reinterpret_cast<SmemB*>(smem_raw);
    const int s = (int)(g % STAGES_B);
    const uint32_t ph = (g / STAGES_B) & 1u;
    const bool landed = sy::bar_wait(&sm.full[s], ph, &sm.abort, err, wait_ns);
    if (!__all_sync(0xffffffffu, landed)) return false;
    if (first_of_item && sm.tile_of[lt_of_g % STAGES_B] < 0) return true;
    const int pc = sm.pcol[s];
    if (pc >= 0) {
#pragma unroll
      for (int rr = 0; rr < ROWS_PER_WARP; ++rr) {
        const int kk = warp * ROWS_PER_WARP + rr;
        const float p = sm.P[s][kk][pc];
        float4* a = reinterpret_cast<float4*>(&sm.A[s][kk][lane * 4]);
        float4 v = *a;
        v.x = fminf(v.x, p);
        v.y = fminf(v.y, p);
        v.z = fminf(v.z, p);
        v.w = fminf(v.w, p);
        *a = v;
      }
      // the TMA refill of this stage comes later through the async proxy
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncwarp();
    if (lane == 0) sy::bar_arrive(&sm.ready[s]);
    return true;
  };

  const mg::Lanes3 L;
  mg::AccMix<C::NJ> acc;  // packed adds for columns 0, 1, scalar for 2, 3 (identical values)
  uint32_t it = 0;
  bool ok = prepare(0, 0, true);
  for (int lt = 0; ok; ++lt) {
    const int t = sm.tile_of[lt % STAGES_B];  // published by the full barrier prepare() waited on
    if (t < 0) break;
    const BatchItem w = items[t];
    const BatchProbTma& pr = probs[w.prob];
    const int nv = pr.nv;
    const int nkb = max(1, (pr.nf + BKB - 1) / BKB);
    int row0, col0, j = -1;
    if (w.kind == BK_TILE3) {
      j = w.a;
      row0 = (w.b >> 16) * C::BM;
      col0 = (w.b & 0xffff) * C::BN;
    } else {
      row0 = w.a * C::BM;
      col0 = w.b * C::BN;
    }
    // 3-way: a warp whose block has no row i < j, no column k > j, or no
    // column inside the matrix skips the min-adds
    const bool active =
        j < 0 || (row0 + L.wrow0 < j && col0 + L.wcol0 + mg::Lanes3::BW - 1 > j && col0 + L.wcol0 < nv);
    acc.zero();
    for (int kb = 0; kb < nkb; ++kb, ++it) {
      if (producer) ok = issue_one();
      ok = __all_sync(0xffffffffu, ok);
      if (ok) ok = prepare(it + 1, kb + 1 == nkb ? lt + 1 : lt, kb + 1 == nkb);
      if (!ok) break;
      const int s = (int)(it % STAGES_B);
      const uint32_t ph = (it / STAGES_B) & 1u;
      const bool prepared = sy::bar_wait(&sm.ready[s], ph, &sm.abort, err, wait_ns);
      if (!__all_sync(0xffffffffu, prepared)) { ok = false; break; }
      if (active) {
        const float* As = &sm.A[s][0][L.am];
        const float* Bs = &sm.B[s][0][L.bn];
#pragma unroll 16
        for (int kk = 0; kk < BKB; ++kk) {
          const float4 a0 = *reinterpret_cast<const float4*>(As + kk * C::BM);
          const float4 a1 = *reinterpret_cast<const float4*>(As + kk * C::BM + mg::Lanes3::RUN);
          const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
          const float4 b0 = *reinterpret_cast<const float4*>(Bs + kk * C::BN);
          const float b[4] = {b0.x, b0.y, b0.z, b0.w};
          acc.step(a, b);
        }
      }
      __syncwarp();
      if (lane == 0) sy::bar_arrive(&sm.empty[s]);
      if ((kb + 1) % FOLD_SLICES == 0) acc.fold();
    }
    if (!ok) break;
    acc.fold();
    if (w.kind == BK_TILE2) {
      mg::store_tile2<C, true, mg::Lanes3>(acc, L, row0, col0, nv, pr.S, pr.out,
                                           pr.out_f64 ? OUT2_C2_F64 : OUT2_C2_F32);
    } else if (w.kind == BK_N2) {
      mg::store_tile2<C, true, mg::Lanes3>(acc, L, row0, col0, nv, pr.S, pr.n2, OUT2_N2_SQUARE_F32);
      __syncwarp();
      if (lane == 0) {
        __threadfence();
        atomicAdd(&n2_done[w.prob], 1);
      }
    } else {
      // Section 2.2 eq. (1) once the problem's n2 table is complete
      if (!warp_wait_count(&n2_done[w.prob], pr.n2_target, &sm.abort, err, wait_ns)) { ok = false; break; }
      const int64_t wdt = nv - 1 - j;
      const int64_t base = mg::slab_offset(nv, 0, j);
      const float Sj = (float)pr.S[j];
      float* out = static_cast<float*>(pr.out);
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int i = row0 + L.row(r);
        if (i >= j) continue;
        const float Sij = __fadd_rn((float)pr.S[i], Sj);
        const float n2ij = __ldcg(pr.n2 + (int64_t)i * nv + j);
#pragma unroll
        for (int c = 0; c < C::NJ; ++c) {
          const int k = col0 + L.col(c);
          if (k <= j || k >= nv) continue;
          out[base + (int64_t)i * wdt + (k - j - 1)] =
              mg::c3_value(acc.hl(r, c), n2ij, __ldcg(pr.n2 + (int64_t)i * nv + k),
                           __ldcg(pr.n2 + (int64_t)j * nv + k), __fadd_rn(Sij, (float)pr.S[k]));
        }
      }
    }
  }
  __syncthreads();
  if (*(volatile int*)&sm.abort) sy::drain_after_abort();
}

// Per-vector FP64 sums of every problem (the same fixed order as
// vector_sums_fm, so the values equal the single-problem path's): block b of
// the grid covers 32 vectors of problem prob_of_block[b].
__global__ void __launch_bounds__(256) batched_sums_kernel(const BatchProbTma* __restrict__ probs,
                                                           const int2* __restrict__ blocks) {
  __shared__ double part[8][33];
  const int2 pb = blocks[blockIdx.x];  // (problem, 32-vector block)
  const BatchProbTma& pr = probs[pb.x];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t i = (int64_t)pb.y * 32 + lane;
  double s = 0.0;
  if (i < pr.nv)
    for (int64_t q = warp; q < pr.nf; q += 8) s += (double)__ldg(pr.V + i + q * pr.ld);
  part[warp][lane] = s;
  __syncthreads();
  if (warp == 0 && i < pr.nv) {
    double t = part[0][lane];
#pragma unroll
    for (int w = 1; w < 8; ++w) t += part[w][lane];
    const_cast<double*>(pr.S)[i] = t;
  }
}

}  // namespace

size_t batched_tma_smem() { return sizeof(SmemB); }

bool make_batch_prob_tma(BatchProbTma* p, const float* V, int64_t nv, int64_t nf, int64_t ld) {
  p->V = V;
  p->ld = ld;
  p->nv = (int)nv;
  p->nf = (int)nf;
  if (nf <= 0) return false;
  return sy::make_map_f32(&p->mapV, V, nv, nf, ld, C::BM, BKB) && sy::make_map_f32(&p->mapP, V, nv, nf, ld, PBOX, BKB);
}

cudaError_t launch_batched_tma(ps_ctx* h, const BatchProbTma* probs, const int2* sum_blocks, int nsum_blocks,
                               const BatchItem* items, int nitems, int* counters, cudaStream_t st) {
  static std::mutex mu;
  static uint64_t attr_done = 0;
  {
    std::lock_guard<std::mutex> lk(mu);
    const uint64_t bit = 1ull << (h->device & 63);
    if (!(attr_done & bit)) {
      const cudaError_t e = cudaFuncSetAttribute(batched_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)sizeof(SmemB));
      if (e != cudaSuccess) return e;
      attr_done |= bit;
    }
  }
  if (nsum_blocks > 0) batched_sums_kernel<<<nsum_blocks, 256, 0, st>>>(probs, sum_blocks);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || nitems == 0) return e;
  const unsigned grid = (unsigned)std::min<int64_t>(nitems, (int64_t)h->num_sms);
  batched_tma_kernel<<<grid, C::NT, sizeof(SmemB), st>>>(probs, items, nitems, counters, h->wait_ns);
  return cudaGetLastError();
}

}  // namespace ps
