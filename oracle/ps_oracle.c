/*
 * ps_oracle.c -- plain FP64 CPU oracle for the Proportional Similarity
 * (Czekanowski) metrics of Joubert, Nance, Weighill and Jacobson,
 * "Parallel Accelerated Vector Similarity Calculations for Genomics
 * Applications" (arXiv 1705.08210).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * statement of what the GPU library computes.  Only the test suite, the
 * package's smoke check and the CPU-baseline leg of the benchmark may load
 * it.  It shares no code, header or table with the CUDA library, and the
 * library never calls it.
 *
 * Everything is evaluated in IEEE double precision with plain loops, in the
 * order the definitions are written.  Build with -ffp-contract=off so that no
 * multiply-add is fused (the compiler default on aarch64 would fuse them).
 *
 * Input layout (this file only): vector-major, element (i,q) = V[i*nf + q],
 * i.e. vector i is the contiguous row V[i*nf .. i*nf+nf-1].
 *
 * Readings where the paper is silent (all of them pinned by tests):
 *   - a pair or triple whose denominator is zero (all-zero vectors) has
 *     metric 0;
 *   - the ratio is evaluated exactly as (2*n2)/(S_i+S_j) and
 *     (1.5*n3)/((S_i+S_j)+S_k), with n3 = ((n2_ij + n2_ik) + n2_jk) - n3';
 *   - 2-way output order: strict upper triangle, row-major,
 *     index(i,j) = i*(2*nv-i-1)/2 + (j-i-1) for i<j;
 *   - 3-way output order: pivot slabs; pivot j owns a j x (nv-1-j) block,
 *     rows i in [0,j), columns k in (j,nv), row-major, blocks in increasing j;
 *   - quantizer: P = the nearest-rank 99.9th percentile of the nonzero
 *     entries (rank r = ceil(0.999*m) of m nonzeros, ascending, 1-based),
 *     level = min(L-1, floor(fl32(fl32(x * r32) + 0.5f))) with
 *     r32 = fl32((L-1)/P), all in IEEE single precision, zero -> level 0.
 *
 * Parity pins: every function below is pinned by tests that do not restate
 * it (Bray-Curtis via scipy, the max-form of the 3-way numerator, sorting
 * identities, Dice/Sorenson set counts, invariants, analytic families).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Number of threads an OpenMP region of this library uses (1 without
 * OpenMP).  Reported by the CPU baseline as its core count. */
int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void oracle_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* Section 2.1: the per-vector sum  S_i = sum_q v_{i,q}.  The 2-way
 * denominator is d2(v_i,v_j) = S_i + S_j and the 3-way denominator
 * (Section 2.2) is d3 = S_i + S_j + S_k. */
void oracle_vector_sums(const double* V, int64_t nv, int64_t nf, double* S) {
  for (int64_t i = 0; i < nv; ++i) {
    double s = 0.0;
    for (int64_t q = 0; q < nf; ++q) s += V[i * nf + q];
    S[i] = s;
  }
}

/* Section 2.1: n2(v_i,v_j) = sum_q min(v_{i,q}, v_{j,q}) (the "min-product"
 * sum). */
double oracle_n2(const double* V, int64_t nf, int64_t i, int64_t j) {
  const double* a = V + i * nf;
  const double* b = V + j * nf;
  double s = 0.0;
  for (int64_t q = 0; q < nf; ++q) s += (a[q] < b[q]) ? a[q] : b[q];
  return s;
}

/* Section 2.2: n3'(v_i,v_j,v_k) = sum_q min(v_{i,q}, v_{j,q}, v_{k,q}). */
double oracle_n3prime(const double* V, int64_t nf, int64_t i, int64_t j,
                      int64_t k) {
  const double* a = V + i * nf;
  const double* b = V + j * nf;
  const double* c = V + k * nf;
  double s = 0.0;
  for (int64_t q = 0; q < nf; ++q) {
    double m = (a[q] < b[q]) ? a[q] : b[q];
    m = (m < c[q]) ? m : c[q];
    s += m;
  }
  return s;
}

/* Section 2.1: c2 = 2 n2 / d2 with d2 = S_i + S_j. */
static double c2_from(double n2, double Si, double Sj) {
  double d = Si + Sj;
  if (d == 0.0) return 0.0;
  return (2.0 * n2) / d;
}

/* Section 2.2, eq. (1): n3 = n2(ij) + n2(ik) + n2(jk) - n3',
 * c3 = (3/2) n3 / d3 with d3 = S_i + S_j + S_k. */
static double c3_from(double n2ij, double n2ik, double n2jk, double n3p,
                      double Si, double Sj, double Sk) {
  double d = (Si + Sj) + Sk;
  if (d == 0.0) return 0.0;
  double n3 = ((n2ij + n2ik) + n2jk) - n3p;
  return (1.5 * n3) / d;
}

double oracle_c2(const double* V, const double* S, int64_t nf, int64_t i,
                 int64_t j) {
  return c2_from(oracle_n2(V, nf, i, j), S[i], S[j]);
}

double oracle_c3(const double* V, const double* S, int64_t nf, int64_t i,
                 int64_t j, int64_t k) {
  return c3_from(oracle_n2(V, nf, i, j), oracle_n2(V, nf, i, k),
                 oracle_n2(V, nf, j, k), oracle_n3prime(V, nf, i, j, k), S[i],
                 S[j], S[k]);
}

/* Position of pair (i,j), i<j, in the packed strict upper triangle. */
static int64_t pair_index(int64_t nv, int64_t i, int64_t j) {
  return i * (2 * nv - i - 1) / 2 + (j - i - 1);
}

/* All n2(v_i,v_j), i<j, packed (Section 2.1, the unique entries of
 * M = V^T min-product V of Section 3.1). */
void oracle_n2_packed(const double* V, int64_t nv, int64_t nf, double* out) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t i = 0; i < nv; ++i)
    for (int64_t j = i + 1; j < nv; ++j)
      out[pair_index(nv, i, j)] = oracle_n2(V, nf, i, j);
}

/* All c2(v_i,v_j), i<j, packed (Section 2.1). */
void oracle_c2_packed(const double* V, int64_t nv, int64_t nf, double* out) {
  double* S = (double*)malloc((size_t)(nv > 0 ? nv : 1) * sizeof(double));
  oracle_vector_sums(V, nv, nf, S);
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t i = 0; i < nv; ++i)
    for (int64_t j = i + 1; j < nv; ++j)
      out[pair_index(nv, i, j)] = oracle_c2(V, S, nf, i, j);
  free(S);
}

/* c2 for an explicit list of pairs (pairs[2p], pairs[2p+1]); used to check
 * sampled outputs of large problems. */
void oracle_c2_pairs(const double* V, int64_t nv, int64_t nf,
                     const int64_t* pairs, int64_t npairs, double* out) {
  double* S = (double*)malloc((size_t)(nv > 0 ? nv : 1) * sizeof(double));
  oracle_vector_sums(V, nv, nf, S);
#pragma omp parallel for schedule(static)
  for (int64_t p = 0; p < npairs; ++p)
    out[p] = oracle_c2(V, S, nf, pairs[2 * p], pairs[2 * p + 1]);
  free(S);
}

/* c3 for an explicit list of triples (t[3p], t[3p+1], t[3p+2]). */
void oracle_c3_triples(const double* V, int64_t nv, int64_t nf,
                       const int64_t* t, int64_t n, double* out) {
  double* S = (double*)malloc((size_t)(nv > 0 ? nv : 1) * sizeof(double));
  oracle_vector_sums(V, nv, nf, S);
#pragma omp parallel for schedule(static)
  for (int64_t p = 0; p < n; ++p)
    out[p] = oracle_c3(V, S, nf, t[3 * p], t[3 * p + 1], t[3 * p + 2]);
  free(S);
}

/* n3' for an explicit list of triples. */
void oracle_n3prime_triples(const double* V, int64_t nf, const int64_t* t,
                            int64_t n, double* out) {
#pragma omp parallel for schedule(static)
  for (int64_t p = 0; p < n; ++p)
    out[p] = oracle_n3prime(V, nf, t[3 * p], t[3 * p + 1], t[3 * p + 2]);
}

/* Number of entries of pivots [j_begin, j_end) in the pivot-slab layout. */
int64_t oracle_slab_size(int64_t nv, int64_t j_begin, int64_t j_end) {
  int64_t n = 0;
  for (int64_t j = j_begin; j < j_end; ++j) n += j * (nv - 1 - j);
  return n;
}

/* All c3(v_i,v_j,v_k), i<j<k, for pivots j in [j_begin, j_end), in the
 * pivot-slab order (Section 2.2 eq. (1); the pivot j plays the role of the
 * column v_j min-ed into X_j in Section 3.2). */
void oracle_c3_slab(const double* V, int64_t nv, int64_t nf, int64_t j_begin,
                    int64_t j_end, double* out) {
  double* S = (double*)malloc((size_t)(nv > 0 ? nv : 1) * sizeof(double));
  oracle_vector_sums(V, nv, nf, S);
  for (int64_t j = j_begin; j < j_end; ++j) {
    int64_t base = oracle_slab_size(nv, j_begin, j);
    int64_t w = nv - 1 - j;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < j; ++i)
      for (int64_t k = j + 1; k < nv; ++k)
        out[base + i * w + (k - j - 1)] = oracle_c3(V, S, nf, i, j, k);
  }
  free(S);
}

/* Thresholded 3-way search: every triple i<j<k with c3 >= tau, in
 * lexicographic (i,j,k) order.  Writes at most `capacity` entries and
 * returns the total count. */
int64_t oracle_threshold_3way(const double* V, int64_t nv, int64_t nf,
                              double tau, int32_t* ijk, double* val,
                              int64_t capacity) {
  double* S = (double*)malloc((size_t)(nv > 0 ? nv : 1) * sizeof(double));
  oracle_vector_sums(V, nv, nf, S);
  int64_t count = 0;
  for (int64_t i = 0; i < nv; ++i)
    for (int64_t j = i + 1; j < nv; ++j)
      for (int64_t k = j + 1; k < nv; ++k) {
        double c = oracle_c3(V, S, nf, i, j, k);
        if (c >= tau) {
          if (count < capacity) {
            ijk[3 * count] = (int32_t)i;
            ijk[3 * count + 1] = (int32_t)j;
            ijk[3 * count + 2] = (int32_t)k;
            val[count] = c;
          }
          ++count;
        }
      }
  free(S);
  return count;
}

/* ---- quantized (thermometer) path: not in the paper; the quantizer
 * reading is stated in the header comment above. ---- */

static int cmp_float(const void* a, const void* b) {
  float x = *(const float*)a, y = *(const float*)b;
  return (x > y) - (x < y);
}

/* Nearest-rank 99.9th percentile of the nonzero entries of x[0..n).
 * Returns 0 when there are no nonzero entries. */
float oracle_percentile_nonzero(const float* x, int64_t n, double p) {
  int64_t m = 0;
  for (int64_t t = 0; t < n; ++t)
    if (x[t] != 0.0f) ++m;
  if (m == 0) return 0.0f;
  float* nz = (float*)malloc((size_t)m * sizeof(float));
  int64_t c = 0;
  for (int64_t t = 0; t < n; ++t)
    if (x[t] != 0.0f) nz[c++] = x[t];
  qsort(nz, (size_t)m, sizeof(float), cmp_float);
  int64_t r = (int64_t)ceil(p * (double)m); /* 1-based rank */
  if (r < 1) r = 1;
  if (r > m) r = m;
  float v = nz[r - 1];
  free(nz);
  return v;
}

/* Uniform quantizer to levels 0..L-1 with the reciprocal scale
 * r32 = fl32((L-1)/P), evaluated in IEEE single precision. */
void oracle_quantize(const float* x, int64_t n, int levels, float P,
                     int32_t* q) {
  volatile float r32 = (float)(levels - 1) / P;
  for (int64_t t = 0; t < n; ++t) {
    float v = x[t];
    if (v == 0.0f || P == 0.0f) {
      q[t] = 0;
      continue;
    }
    volatile float prod = v * r32;
    volatile float shifted = prod + 0.5f;
    float f = floorf(shifted);
    /* min(L-1, .) taken before the integer conversion, which is undefined
     * for values beyond the int32 range */
    int32_t l = (f >= (float)(levels - 1)) ? levels - 1 : (int32_t)f;
    if (l < 0) l = 0;
    q[t] = l;
  }
}
