// hmat_kernels.cu -- device side of the H-matrix library (sm_103a).
//
//  * exec_tasks: one persistent kernel that runs a dependency-ordered task
//    list (the unrolled H-LU / H-solve / H x thin-dense recursions).  CTAs take
//    tasks in list order from a global counter; a task waits (bounded, acquire
//    loads) until its predecessors are marked done, runs on the whole CTA, and
//    marks itself done with a release store.  Because tasks are taken in a
//    topological order and every CTA of the grid is resident, the lowest
//    unfinished task always has its predecessors finished: no deadlock.  A
//    wait that exceeds its limit writes HMAT_ERR_TIMEOUT into the status word;
//    once the status is non-zero every remaining task is skipped and marked
//    done, so the kernel always terminates.
//  * trunc_batched: Section 3 "Truncation" of independent low-rank matrices,
//    one CTA each.
//  * csr_scatter / to_dense: H-matrix construction and dense export.
#include <cuda_runtime.h>
#include <stdint.h>

#include "hmat_device.cuh"
#include "hmat_kernels.h"
#include "hmat_mlp.cuh"

namespace hm {

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Locations: bits 60-61 select the base (0 H storage, 1 workspace, 2 and 3
// caller buffers), the rest is an offset in doubles.
__device__ __forceinline__ double* loc(const ExecEnv& e, int64_t l) {
  if (l < 0) return nullptr;
  int64_t off = l & ((WS_BIT)-1);
  switch ((int)((l >> 60) & 3)) {
    case 0: return e.hbase + off;
    case 1: return e.wsbase + off;
    case 2: return e.ext0 + off;
    default: return e.ext1 + off;
  }
}
__device__ __forceinline__ int width_of(const ExecEnv& e, int w) { return w >= 0 ? w : e.ranks[-w - 1]; }

// true iff every entry of the m x n matrix (ld) is zero
__device__ bool cta_all_zero(const double* A, int ld, int m, int n, Smem& s) {
  int nz = 0;
  for (int idx = threadIdx.x; idx < m * n; idx += HM_THREADS)
    if (A[(int64_t)(idx / m) * ld + idx % m] != 0.0) nz = 1;
  nz = __syncthreads_or(nz);
  return !nz;
}

__device__ void cta_copy(double* C, int ldc, const double* A, int lda, int m, int n, bool trans, double alpha) {
  for (int idx = threadIdx.x; idx < m * n; idx += HM_THREADS) {
    int i = idx % m, j = idx / m;
    double v = trans ? A[(int64_t)i * lda + j] : A[(int64_t)j * lda + i];
    C[(int64_t)j * ldc + i] = alpha * v;
  }
}

// true iff U (m x k) and V (n x k) hold only finite numbers
__device__ bool cta_finite(const double* U, int ldu, int m, int k, const double* V, int ldv, int n) {
  int bad = 0;
  for (int idx = threadIdx.x; idx < m * k; idx += HM_THREADS)
    if (!isfinite(U[(int64_t)(idx / m) * ldu + idx % m])) bad = 1;
  for (int idx = threadIdx.x; idx < n * k; idx += HM_THREADS)
    if (!isfinite(V[(int64_t)(idx / n) * ldv + idx % n])) bad = 1;
  return !__syncthreads_or(bad);
}

// first randomised truncation whose result was not finite (it is then redone
// by the exact path): path, m, n, l, k, scale
__device__ void record_bad(const ExecEnv& e, int path, int m, int n, int l, int k, double scale) {
  if (threadIdx.x == 0 && atomicCAS(e.counters + 3, 0ull, (unsigned long long)path) == 0ull) {
    e.counters[4] = (unsigned long long)m;
    e.counters[5] = (unsigned long long)n;
    e.counters[6] = (unsigned long long)l;
    e.counters[7] = (unsigned long long)k;
    e.counters[8] = __double_as_longlong(scale);
  }
}

// First sketch width of a randomised truncation: kz + 6 (at least 8), kz the
// larger input rank, without a predictor; else max(predicted rank + 3, kz + 2).
// l is the total input rank (a feature of the predictor).
// One term SA SB^T of an explicit M, placed at columns [c0, c0 + n).
struct M32Part {
  const double* SA;  // m x k (ld m)
  const double* SB;  // n x k (ld n)
  int k, n, c0;
};

// Mixed path: M = base + sum of the parts, formed as M / S in FP32 (M32
// holds m x ncol floats, ld m).  The factors are converted once to FP32,
// scaled so that every product and the base stay below 1 in magnitude
// (S = max(max|SA| max|SB|, max|base|)); the products accumulate in FP32.
// fac: sum over parts of (m + n) k floats.  Returns 0 with *S set, or 1 if
// the result is not finite, or 2 if the terms cancel so much that FP32
// rounding of the sum could reach eps ||M||_F / 10 (the caller then uses
// the exact FP64 path).
template <class Base>
__device__ int form_m32(int m, int ncol, const M32Part* P, int np, bool has_base, Base base, float* M32,
                        float* fac, double eps, double* S_out, Smem& s) {
  int tid = threadIdx.x;
  double ma = 0.0, mb = 0.0, mz = 0.0;
  for (int q = 0; q < np; ++q) {
    for (int idx = tid; idx < m * P[q].k; idx += HM_THREADS) ma = fmax(ma, fabs(P[q].SA[idx]));
    for (int idx = tid; idx < P[q].n * P[q].k; idx += HM_THREADS) mb = fmax(mb, fabs(P[q].SB[idx]));
  }
  if (has_base)
    for (int idx = tid; idx < m * ncol; idx += HM_THREADS) mz = fmax(mz, fabs(base(idx % m, idx / m)));
  ma = block_max(ma, s);
  mb = block_max(mb, s);
  mz = block_max(mz, s);
  double S = fmax(ma * mb, mz);
  *S_out = S;
  if (!isfinite(S)) return 1;
  if (S == 0.0) {
    for (int idx = tid; idx < m * ncol; idx += HM_THREADS) M32[idx] = 0.f;
    __syncthreads();
    return 0;
  }
  double sa = ma > 0.0 ? 1.0 / ma : 0.0, sb = ma / S, sz = 1.0 / S;
  float* fa[2];
  float* fb[2];
  float* f = fac;
  for (int q = 0; q < np; ++q) {
    fa[q] = f;
    fb[q] = f + (int64_t)m * P[q].k;
    f = fb[q] + (int64_t)P[q].n * P[q].k;
    for (int idx = tid; idx < m * P[q].k; idx += HM_THREADS) fa[q][idx] = (float)(P[q].SA[idx] * sa);
    for (int idx = tid; idx < P[q].n * P[q].k; idx += HM_THREADS) fb[q][idx] = (float)(P[q].SB[idx] * sb);
  }
  __syncthreads();
  float sm = 0.f, sabs = 0.f;
  for (int idx = tid; idx < m * ncol; idx += HM_THREADS) {
    int i = idx % m, c = idx / m;
    float v = has_base ? (float)(base(i, c) * sz) : 0.f;
    float a = fabsf(v);
    for (int q = 0; q < np; ++q) {
      int cc = c - P[q].c0;
      if (cc < 0 || cc >= P[q].n) continue;
      const float* pa = fa[q] + i;
      const float* pb = fb[q] + cc;
      for (int j = 0; j < P[q].k; ++j) {
        float x = pa[(int64_t)j * m] * pb[(int64_t)j * P[q].n];
        v += x;
        a += fabsf(x);
      }
    }
    M32[idx] = v;
    sm += v * v;
    sabs += a * a;
  }
  double tm = block_sum((double)sm, s), ta = block_sum((double)sabs, s);
  {
    double f = 0.0;
    for (int q = 0; q < np; ++q) f += 2.0 * m * (double)P[q].n * P[q].k;
    count_f32(s, f);
  }
  if (!isfinite(tm) || !isfinite(ta)) return 1;
  // FP32 rounding of the sums stays below ~3e-7 ||terms||_F (terms: the
  // entrywise sums of magnitudes); keep it under eps ||M||_F / 10
  if (ta * 9e-14 > 1e-2 * eps * eps * tm) return 2;
  return 0;
}

__device__ int sketch_width(const ExecEnv& e, long long ti, int kz, int l, Smem& s) {
  if (!e.mlp) {
    int r0 = kz + 6;
    return r0 < 8 ? 8 : r0;
  }
  if ((threadIdx.x >> 5) == 0) {
    float x[HM_MLP_IN];
    for (int i = 0; i < 4; ++i) x[i] = e.feat[4 * ti + i];
    x[4] = (float)l / 16.f;
    x[5] = (float)log10(e.eps) / 4.f;
    float y = mlp_forward_warp((const __nv_bfloat16*)e.mlp, x);
    if ((threadIdx.x & 31) == 0) s.bcast[1] = (double)y;
  }
  __syncthreads();
  double y = s.bcast[1];
  __syncthreads();
  double kh = expm1(y < 8.0 ? y : 8.0);
  if (kh < 0.0) kh = 0.0;
  // never below kz + 2: a truncated sum rarely loses rank against its larger
  // term, and a sketch that misses costs a second, doubled one
  int r0 = (int)ceil(kh) + e.oversample;
  if (r0 < kz + 2) r0 = kz + 2;
  return r0 < 2 ? 2 : r0;
}

// Training pair of an exact truncation: features and log(1 + rank); l is the
// total input rank.
__device__ void record_rank(const ExecEnv& e, long long ti, int l, int k) {
  if (!e.rec || threadIdx.x != 0) return;
  unsigned long long i = atomicAdd(e.rec_count, 1ull);
  if ((long long)i >= e.rec_cap) return;
  float* r = e.rec + 7 * i;
  for (int j = 0; j < 4; ++j) r[j] = e.feat[4 * ti + j];
  r[4] = (float)l / 16.f;
  r[5] = (float)log10(e.eps) / 4.f;
  r[6] = (float)log1p((double)k);
}

// attempts and columns sketched (over all attempts) by a randomised
// truncation; with task profiling also the task's note: stacked width l
// (bits 0-11), path (12-14: 1 FP32 randomised, 2 FP64 randomised, 3 exact),
// a failed randomised attempt before the exact one (bit 15), rank (16-23),
// sketch attempts (24-31).  path 0 = the randomised truncation failed.
__device__ void count_sketch(const ExecEnv& e, Smem& s, long long ti, int l, int path, int k) {
  if (threadIdx.x == 0) {
    atomicAdd(e.counters + 9, (unsigned long long)s.ivals[5]);
    atomicAdd(e.counters + 10, (unsigned long long)s.ivals[6]);
    if (e.task_aux) {
      unsigned att = (unsigned)(s.ivals[5] < 255 ? s.ivals[5] : 255) << 24;
      e.task_aux[ti] = path ? ((unsigned)(l < 4095 ? l : 4095) | ((unsigned)path << 12) |
                               ((unsigned)(k < 255 ? k : 255) << 16) | att)
                            : (0x8000u | att);
    }
  }
}
__device__ void note_exact(const ExecEnv& e, long long ti, int l, int k) {
  if (threadIdx.x == 0 && e.task_aux)
    e.task_aux[ti] = (e.task_aux[ti] & 0xFF008000u) | (unsigned)(l < 4095 ? l : 4095) | (3u << 12) |
                     ((unsigned)(k < 255 ? k : 255) << 16);
}

// ---------------------------------------------------------------------------
// Task bodies
// ---------------------------------------------------------------------------
// Inverse of a dense diagonal leaf (H-inversion, leaf case of Fig. invert):
// no-pivot LU and two triangular solves on the identity, in shared memory
// (2 n^2 <= HM_JAC_SMEM doubles, n <= 67; larger leaves set DS_INTERNAL).
__device__ void task_inv(const ExecEnv& e, const HTask& t, Smem& s) {
  int n = t.m;
  if (2 * (int64_t)n * n > HM_JAC_SMEM) {
    if (threadIdx.x == 0) set_status(e.status, DS_INTERNAL);
    return;
  }
  double* A = loc(e, t.a);
  double* As = s.jac;
  double* X = s.jac + (int64_t)n * n;
  for (int idx = threadIdx.x; idx < n * n; idx += HM_THREADS) {
    As[idx] = A[(int64_t)(idx / n) * t.lda + idx % n];
    X[idx] = (idx % n == idx / n) ? 1.0 : 0.0;
  }
  __syncthreads();
  cta_lu(As, n, n, e.status);
  __syncthreads();
  if (threadIdx.x == 0) s.ivals[11] = ld_acquire(e.status);  // one decision for the whole CTA
  __syncthreads();
  if (s.ivals[11] != 0) return;
  cta_trsm_cols(TRSM_L, As, n, n, X, n, n);
  cta_trsm_cols(TRSM_U, As, n, n, X, n, n);
  for (int idx = threadIdx.x; idx < n * n; idx += HM_THREADS) A[(int64_t)(idx / n) * t.lda + idx % n] = X[idx];
  __syncthreads();
}

// Cholesky of a dense SPD diagonal leaf (H-Cholesky, leaf case): the lower
// factor L in the lower triangle, L^T mirrored into the strictly upper one,
// right-looking in shared memory (n^2 <= HM_JAC_SMEM doubles, n <= 96;
// larger leaves set DS_INTERNAL).  A non-positive pivot sets DS_SINGULAR.
__device__ void task_chol(const ExecEnv& e, const HTask& t, Smem& s) {
  int n = t.m;
  if ((int64_t)n * n > HM_JAC_SMEM) {
    if (threadIdx.x == 0) set_status(e.status, DS_INTERNAL);
    return;
  }
  double* A = loc(e, t.a);
  double* As = s.jac;
  for (int idx = threadIdx.x; idx < n * n; idx += HM_THREADS) As[idx] = A[(int64_t)(idx / n) * t.lda + idx % n];
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x == 0) {
      double d = As[k + (int64_t)k * n];
      s.ivals[11] = (d > 0.0 && isfinite(d)) ? 0 : 1;
      if (s.ivals[11]) set_status(e.status, DS_SINGULAR);
      s.bcast[0] = s.ivals[11] ? 1.0 : sqrt(d);
    }
    __syncthreads();
    if (s.ivals[11]) return;  // the same decision on every thread
    double lkk = s.bcast[0];
    double inv = 1.0 / lkk;
    for (int i = k + 1 + threadIdx.x; i < n; i += HM_THREADS) As[i + (int64_t)k * n] *= inv;
    __syncthreads();
    if (threadIdx.x == 0) As[k + (int64_t)k * n] = lkk;
    int rem = n - k - 1;
    for (int idx = threadIdx.x; idx < rem * rem; idx += HM_THREADS) {
      int i = k + 1 + idx % rem, j = k + 1 + idx / rem;
      if (j <= i) As[i + (int64_t)j * n] -= As[i + (int64_t)k * n] * As[j + (int64_t)k * n];
    }
    __syncthreads();
  }
  for (int idx = threadIdx.x; idx < n * n; idx += HM_THREADS) {
    int i = idx % n, j = idx / n;
    A[(int64_t)j * t.lda + i] = i >= j ? As[i + (int64_t)j * n] : As[j + (int64_t)i * n];
  }
  __syncthreads();
}

__device__ void task_hmv(const ExecEnv& e, const HTask& t, Smem& s, bool f32) {
  bool trans = t.flags & F_TRANS;
  int w = width_of(e, t.wa);
  double* out = loc(e, t.c);
  const double* in = loc(e, t.b);
  if (t.flags & F_ZERO_OUT) {
    // a gang member zeroes its own rows [p, q) of the output
    int z0 = t.pad1 > 1 ? t.p : 0, zr = (t.pad1 > 1 ? t.q : t.m) - z0;
    for (int idx = threadIdx.x; idx < zr * w; idx += HM_THREADS)
      out[(int64_t)(idx / zr) * t.ldc + z0 + idx % zr] = 0.0;
    __syncthreads();
  }
  if (w <= 0) return;
  for (int li = 0; li < t.list_len; ++li) {
    const LeafRef L = e.leaves[t.list_begin + li];
    int orow = trans ? L.coff : L.roff;
    int irow = trans ? L.roff : L.coff;
    int orows = trans ? L.cols : L.rows;
    int irows = trans ? L.rows : L.cols;
    if (L.kind == 1) {
      const double* N = loc(e, L.a);
      if (f32) {
        cta_gemm32(out + orow, t.ldc, orows, w, irows, t.alpha, N, L.lda, trans, in + irow, t.ldb, false, false,
                   (float*)s.jac);
        count_f32(s, 2.0 * orows * (double)irows * w);
      } else {
        cta_gemm(out + orow, t.ldc, orows, w, irows, t.alpha, N, L.lda, trans, in + irow, t.ldb, false, false);
        __syncthreads();
      }
    } else if (f32) {
      int k = e.ranks[L.rank_slot];
      if (k <= 0) continue;
      const double* Fin = loc(e, trans ? L.a : L.b);
      const double* Fout = loc(e, trans ? L.b : L.a);
      int ldin = trans ? L.lda : L.ldb;
      int ldout = trans ? L.ldb : L.lda;
      float* zf = (float*)s.jac + HM_G32_SMEM;  // Zhat (k x wc) in FP32
      int wc = (2 * HM_JAC_SMEM - HM_G32_SMEM) / k;
      if (wc > w) wc = w;
      for (int c0 = 0; c0 < w; c0 += wc) {
        int cw = w - c0 < wc ? w - c0 : wc;
        cta_gemm32(zf, k, k, cw, irows, t.alpha, Fin, ldin, true, in + irow + (int64_t)c0 * t.ldb, t.ldb, false,
                   true, (float*)s.jac);
        cta_gemm32(out + orow + (int64_t)c0 * t.ldc, t.ldc, orows, cw, k, 1.0, Fout, ldout, false, zf, k, false,
                   false, (float*)s.jac);
        count_f32(s, 2.0 * (double)k * cw * (irows + orows));
      }
    } else {
      int k = e.ranks[L.rank_slot];
      if (k <= 0) continue;
      const double* Fin = loc(e, trans ? L.a : L.b);   // factor multiplying the input
      const double* Fout = loc(e, trans ? L.b : L.a);  // factor producing the output
      int ldin = trans ? L.lda : L.ldb;
      int ldout = trans ? L.ldb : L.lda;
      // chunk the columns so that Zhat (k x wc) fits in shared memory
      int wc = HM_JAC_SMEM / k;
      if (wc > w) wc = w;
      for (int c0 = 0; c0 < w; c0 += wc) {
        int cw = w - c0 < wc ? w - c0 : wc;
        cta_gemm(s.jac, k, k, cw, irows, t.alpha, Fin, ldin, true, in + irow + (int64_t)c0 * t.ldb, t.ldb, false,
                 true);
        __syncthreads();
        cta_gemm(out + orow + (int64_t)c0 * t.ldc, t.ldc, orows, cw, k, 1.0, Fout, ldout, false, s.jac, k, false,
                 false);
        __syncthreads();
      }
    }
  }
}

__device__ void task_densify(const ExecEnv& e, const HTask& t, Smem& s) {
  bool trans = t.flags & F_TRANS;
  double* out = loc(e, t.c);
  for (int li = 0; li < t.list_len; ++li) {
    const LeafRef L = e.leaves[t.list_begin + li];
    int orow = trans ? L.coff : L.roff;
    int ocol = trans ? L.roff : L.coff;
    int orows = trans ? L.cols : L.rows;
    int ocols = trans ? L.rows : L.cols;
    double* o = out + orow + (int64_t)ocol * t.ldc;
    if (L.kind == 1) {
      cta_copy(o, t.ldc, loc(e, L.a), L.lda, orows, ocols, trans, 1.0);
    } else {
      int k = e.ranks[L.rank_slot];
      const double* U = loc(e, L.a);
      const double* V = loc(e, L.b);
      if (!trans) cta_gemm(o, t.ldc, orows, ocols, k, 1.0, U, L.lda, false, V, L.ldb, true, true);
      else cta_gemm(o, t.ldc, orows, ocols, k, 1.0, V, L.ldb, false, U, L.lda, true, true);
    }
    __syncthreads();
  }
}

// FP32 factored truncation inside a task (trunc_fact32): SA (m x l) and SB
// (n x l, or two diagonal blocks n0 x k0 and n1 x k1 when sb1 is given) are
// copied to FP32, scaled by their largest entries.  Returns the rank; *ok = 0
// when the caller must fall back to the exact truncation.
__device__ int task_fact32(const ExecEnv& e, const HTask& t, Smem& s, int m, int n, int l, const double* SA,
                           const double* SB0, int n0, int k0, const double* SB1, int n1, int k1, double* ws,
                           uint64_t seed, int r0, double* f, int* ok) {
  double S = 0.0;
  int k = fact32_run(m, n, l, SA, SB0, n0, k0, SB1, n1, k1, ws, e.eps, t.cap, loc(e, t.e), t.lde, loc(e, t.f), t.ldf,
                     e.status, s, seed, r0, f, ok, &S);
  if (*ok && !cta_finite(loc(e, t.e), t.lde, m, k, loc(e, t.f), t.ldf, n)) {
    *ok = 0;
    record_bad(e, 11, m, n, l, k, S);
  }
  return k;
}

// ---------------------------------------------------------------------------
// Gang truncation: one large rkadd of the mixed form run by G CTAs together.
// A single CTA is latency-bound on a 1024 x 1024 or 4096 x 4096 block (every
// Householder step sweeps its whole panel); here every CTA takes its own row
// blocks of the stacked factors and the thin QRs are TSQRs (Demmel, Grigori,
// Hoemmen and Langou, SIAM J. Sci. Comput. 2012): a Householder QR of each
// row block, then one of the stacked l x l R factors, repeated by every
// member.  The steps are those of Fig. rkadd with the FP32 core of the mixed
// form: SB = Q_B R_B, Mhat = SA R_B^T, Mhat = Q_T R_T, the core on R_T, C =
// Q_T (core vectors), D = Q_B (core weights) S.  The members meet at five
// gang barriers (a counter per task, bounded waits); any case the gang does
// not cover (a zero product, a stacked width the stacks cannot hold, a failed
// cancellation guard, a non-finite result) is left to member 0, which runs the
// single-CTA task on the untouched inputs.
// ---------------------------------------------------------------------------
// Arrive at gang barrier k (1-based) of the gang whose member 0 is task c0
// and wait for all G members.
__device__ void gang_sync(const ExecEnv& e, long long c0, int k, int G) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int* ctr = e.gang + c0;
    __threadfence();
    atomicAdd(ctr, 1);
    uint64_t t0 = global_ns();
    long long it = 0;
    while (ld_acquire(ctr) < k * G) {
      if (++it > e.spin_iters || global_ns() - t0 > e.spin_ns) {
        set_status(e.status, DS_TIMEOUT);
        break;
      }
      __nanosleep(32);
    }
    __threadfence();
  }
  __syncthreads();
}

// A member that leaves before barrier `last` arrives at the ones it skips.
__device__ void gang_leave(const ExecEnv& e, long long c0, int passed, int last) {
  __syncthreads();
  if (threadIdx.x == 0 && last > passed) {
    __threadfence();
    atomicAdd(e.gang + c0, last - passed);
  }
  __syncthreads();
}

// The gang region of a task (doubles from the task's scratch base + offset).
struct GangWs {
  double* xch;     // G x HM_GANG_XCH
  float* RB;       // G x L x L: R of every member's block of SB
  float* RM;       // G x L x L: R of every member's block of Mhat
  float* SAf;      // m x L (ld m): FP32 SA, later C's rows
  float* SBf;      // n x L (ld n): FP32 SB, then its blocks' reflectors
  float* Mh;       // m x L (ld m): Mhat, then its blocks' reflectors
  float* Vs;       // n x L (ld n): D's rows
  double* tloc;    // G x 4L: tau and R diagonal of the member's two block QRs
  float* stk;      // G x (3 G L L + L L): every member's two stacks and small panels
  double* tstk;    // G x 4L: tau and R diagonal of the member's two stack QRs
};

__device__ GangWs gang_ws(double* base, int m, int n, int L, int G) {
  GangWs g;
  g.xch = base;
  float* f = (float*)(base + (int64_t)G * HM_GANG_XCH);
  g.RB = f;
  g.RM = g.RB + (int64_t)G * L * L;
  g.SAf = g.RM + (int64_t)G * L * L;
  g.SBf = g.SAf + (int64_t)m * L;
  g.Mh = g.SBf + (int64_t)n * L;
  g.Vs = g.Mh + (int64_t)m * L;
  g.stk = g.Vs + (int64_t)n * L;
  int64_t fl = (int64_t)(g.stk - f) + (int64_t)G * (3 * (int64_t)G * L * L + (int64_t)L * L);
  double* d = (double*)f + (fl + 1) / 2;
  g.tloc = d;
  g.tstk = d + (int64_t)G * 4 * L;
  return g;
}

// Stack the G members' l x l R factors (blocks of R, ld L) into stk (G l x l,
// ld G l) and factor it; returns nothing, the R factor stays in stk's upper
// triangle with its diagonal in rd.
__device__ void gang_stack_qr(const float* R, int G, int l, int L, float* stk, double* tau, double* rd, Smem& s) {
  int gl = G * l;
  for (int idx = threadIdx.x; idx < gl * l; idx += HM_THREADS) {
    int row = idx % gl, c = idx / gl;
    int q = row / l, i = row % l;
    stk[idx] = R[(int64_t)q * L * L + i + (int64_t)c * L];
  }
  cta_qr_rows<float>(stk, gl, gl, l, tau, rd, s);
}

// R (l x l, ld L) of a QR held as reflectors in X (ld ldx) and diagonal rd.
__device__ void gang_put_r(const float* X, int ldx, const double* rd, int l, float* R, int L) {
  for (int idx = threadIdx.x; idx < l * l; idx += HM_THREADS) {
    int i = idx % l, c = idx / l;
    R[i + (int64_t)c * L] = c < i ? 0.f : (c == i ? (float)rd[i] : X[i + (int64_t)c * ldx]);
  }
}

__device__ void task_rkadd(const ExecEnv& e, const HTask& t, Smem& s, long long ti);

__device__ void task_rowmerge(const ExecEnv& e, const HTask& t, Smem& s, long long ti);

// The single-CTA task a gang's member 0 falls back to (a rowmerge gang keeps
// L in q, the single task its second part's rows).
__device__ void gang_fallback(const ExecEnv& e, const HTask& t, Smem& s, long long ti) {
  if (t.type == T_ROWMERGE) {
    HTask u = t;
    u.q = t.n - t.p;
    task_rowmerge(e, u, s, ti);
  } else {
    task_rkadd(e, t, s, ti);
  }
}

// A gang truncation of M = SA SB^T: for T_RKADD SA = [alpha A | Uin], SB =
// [B | Vin] (Fig. rkadd); for T_ROWMERGE SA = [U0 | U1] and SB =
// blockdiag(V0, V1) (Fig. rowmerge: two blocks side by side, n = n0 + n1
// with n0 in p).
__device__ void task_rkadd_gang(const ExecEnv& e, const HTask& t, Smem& s, long long ti) {
  const int r = t.pad0, G = t.pad1, L = t.q;
  const long long c0 = ti - r;  // member 0: the gang's counter
  const int m = t.m, n = t.n, tid = threadIdx.x;
  const bool merge = t.type == T_ROWMERGE;
  const int n0 = merge ? t.p : n;
  const double alpha = merge ? 1.0 : t.alpha;
  bool btr = !merge && (t.flags & F_B_TRANS);
  int w = width_of(e, t.wa);
  int kin = merge ? width_of(e, t.wb) : (t.rin >= 0 ? e.ranks[t.rin] : 0);
  int l = w + kin;
  const double* A = loc(e, t.a);
  const double* B = loc(e, t.b);
  const double* Uin = loc(e, t.c);
  const double* Vin = loc(e, t.d);
  GangWs g = gang_ws(loc(e, t.ws) + t.list_begin, m, n, L, G);
  int mb = (m + G - 1) / G, nb = (n + G - 1) / G;
  int ra = r * mb, rm = min(m, ra + mb) - ra;  // this member's rows of SA / Mhat / C
  int ca = r * nb, rn = min(n, ca + nb) - ca;  // and of SB / D
  auto sa = [&](int i, int j) -> double {    // stacked [alpha A | Uin]
    return j < w ? alpha * A[(int64_t)j * t.lda + i] : Uin[(int64_t)(j - w) * t.ldc + i];
  };
  auto sb = [&](int i, int j) -> double {    // stacked [B | Vin], or blockdiag(B, Vin)
    if (merge) {
      if (j < w) return i < n0 ? B[(int64_t)j * t.ldb + i] : 0.0;
      return i >= n0 ? Vin[(int64_t)(j - w) * t.ldd + i - n0] : 0.0;
    }
    return j < w ? (btr ? B[(int64_t)i * t.ldb + j] : B[(int64_t)j * t.ldb + i]) : Vin[(int64_t)(j - w) * t.ldd + i];
  };
  // 1. the largest entries and the non-zero pattern of this member's rows
  double ma = 0.0, mbx = 0.0;
  int nza = 0, nzb = 0;
  if (l <= L) {
    for (int idx = tid; idx < rm * l; idx += HM_THREADS) {
      double v = sa(ra + idx % rm, idx / rm);
      ma = fmax(ma, fabs(v));
      if (idx / rm < w && v != 0.0) nza = 1;
    }
    for (int idx = tid; idx < rn * l; idx += HM_THREADS) {
      double v = sb(ca + idx % rn, idx / rn);
      mbx = fmax(mbx, fabs(v));
      if (idx / rn < w && v != 0.0) nzb = 1;
    }
  }
  ma = block_max(ma, s);
  mbx = block_max(mbx, s);
  nza = __syncthreads_or(nza);
  nzb = __syncthreads_or(nzb);
  if (tid == 0) {
    double* x = g.xch + (int64_t)r * HM_GANG_XCH;
    x[0] = ma;
    x[1] = mbx;
    x[2] = nza;
    x[3] = nzb;
  }
  gang_sync(e, c0, 1, G);
  // 2. the same decision on every member
  double MA = 0.0, MB = 0.0;
  bool any_a = false, any_b = false;
  for (int q = 0; q < G; ++q) {
    const double* x = g.xch + (int64_t)q * HM_GANG_XCH;
    MA = fmax(MA, x[0]);
    MB = fmax(MB, x[1]);
    any_a = any_a || x[2] != 0.0;
    any_b = any_b || x[3] != 0.0;
  }
  double S = MA * MB;
  bool zero = merge ? (w == 0 || kin == 0) : (w == 0 || ((t.flags & F_CHECK_ZERO) && !(any_a && any_b)));
  bool ok = !zero && l <= L && l <= HM_FACT32_DIRECT && l >= e.rand_min_l && l <= rm && l <= rn && l <= m &&
            l <= n && 3 * (int64_t)l * l + 2 * l <= 2 * (int64_t)HM_JAC_SMEM && S > 0.0 &&
            isfinite(S);
  if (!ok) {
    gang_leave(e, c0, 1, 5);
    if (r == 0) gang_fallback(e, t, s, ti);
    return;
  }
  // 3. FP32 copies of this member's rows, scaled by the largest entries
  {
    double ia = 1.0 / MA, ib = 1.0 / MB;
    for (int idx = tid; idx < rm * l; idx += HM_THREADS) {
      int i = idx % rm, j = idx / rm;
      g.SAf[(int64_t)j * m + ra + i] = (float)(sa(ra + i, j) * ia);
    }
    for (int idx = tid; idx < rn * l; idx += HM_THREADS) {
      int i = idx % rn, j = idx / rn;
      g.SBf[(int64_t)j * n + ca + i] = (float)(sb(ca + i, j) * ib);
    }
  }
  double* tauB = g.tloc + (int64_t)r * 4 * L;
  double* rdB = tauB + L;
  double* tauM = rdB + L;
  double* rdM = tauM + L;
  float* stkB = g.stk + (int64_t)r * (3 * (int64_t)G * L * L + (int64_t)L * L);  // G l x l, ld G l
  float* stkM = stkB + (int64_t)G * L * L;                                        // G l x l, ld G l
  float* Ys = stkM + (int64_t)G * L * L;                                          // G l x k, ld G l
  float* Xs = Ys + (int64_t)G * L * L;                                            // l x k, ld l
  double* tsB = g.tstk + (int64_t)r * 4 * L;
  double* rsB = tsB + L;
  double* tsM = rsB + L;
  double* rsM = tsM + L;
  // 4. QR of this member's block of SB; its R to the exchange
  cta_qr_rows<float>(g.SBf + ca, n, rn, l, tauB, rdB, s);
  gang_put_r(g.SBf + ca, n, rdB, l, g.RB + (int64_t)r * L * L, L);
  gang_sync(e, c0, 2, G);
  // 5. R_B from the stacked R factors; Mhat = SA R_B^T on this member's rows,
  //    with the sums of the cancellation guard; QR of its block
  gang_stack_qr(g.RB, G, l, L, stkB, tsB, rsB, s);
  const int gl = G * l;
  float smm = 0.f, sab = 0.f;
  for (int idx = tid; idx < rm * l; idx += HM_THREADS) {
    int i = idx % rm, c = idx / rm;
    float v = 0.f, a = 0.f;
    for (int j = c; j < l; ++j) {
      float rcj = j == c ? (float)rsB[c] : stkB[c + (int64_t)j * gl];
      float x = g.SAf[(int64_t)j * m + ra + i] * rcj;
      v += x;
      a += fabsf(x);
    }
    g.Mh[(int64_t)c * m + ra + i] = v;
    smm += v * v;
    sab += a * a;
  }
  double tm = block_sum((double)smm, s), ta = block_sum((double)sab, s);
  cta_qr_rows<float>(g.Mh + ra, m, rm, l, tauM, rdM, s);
  gang_put_r(g.Mh + ra, m, rdM, l, g.RM + (int64_t)r * L * L, L);
  if (tid == 0) {
    double* x = g.xch + (int64_t)r * HM_GANG_XCH;
    x[4] = tm;
    x[5] = ta;
  }
  gang_sync(e, c0, 3, G);
  double TM = 0.0, TA = 0.0;
  for (int q = 0; q < G; ++q) {
    TM += g.xch[(int64_t)q * HM_GANG_XCH + 4];
    TA += g.xch[(int64_t)q * HM_GANG_XCH + 5];
  }
  if (!isfinite(TM) || !isfinite(TA) || TA * 9e-14 > 1e-2 * e.eps * e.eps * TM) {
    gang_leave(e, c0, 3, 5);
    if (r == 0) gang_fallback(e, t, s, ti);
    return;
  }
  // 6. R_T from the stacked R factors of Mhat; the FP32 core on R_T (in
  //    shared memory: R_T, then the core's W, Vrot, norms and permutation)
  gang_stack_qr(g.RM, G, l, L, stkM, tsM, rsM, s);
  float* J = (float*)s.jac;
  float* cw = J + l * l;
  for (int idx = tid; idx < l * l; idx += HM_THREADS) {
    int i = idx % l, c = idx / l;
    J[idx] = c < i ? 0.f : (c == i ? (float)rsM[i] : stkM[i + (int64_t)c * gl]);
  }
  __syncthreads();
  core_f32(J, l, l, cw, s, HM_CORE_SWEEPS);
  if (tid == 0) {
    double total = 0.0;
    for (int i = 0; i < l; ++i) total += s.sigma[i] * s.sigma[i];
    double bound = e.eps * e.eps * total, tail = 0.0;
    int k = l;
    while (k > 0) {
      double x = s.sigma[s.order[k - 1]];
      if (tail + x * x <= bound) {
        tail += x * x;
        --k;
      } else {
        break;
      }
    }
    s.ivals[13] = k > t.cap ? 1 : 0;
    s.ivals[4] = k > t.cap ? t.cap : k;
  }
  __syncthreads();
  const int k = s.ivals[4];
  const float* W = cw;
  const float* Vrot = cw + l * l;
  const int* perm = (const int*)(cw + 2 * l * l + l);
  // 7. C = Q_T Q_c Vrot(:, order): the core's reflectors (in J) on the kept
  //    rotation columns, then the stack's reflectors, then this member's
  //    block reflectors; D = Q_B P W(:, order) S likewise
  for (int idx = tid; idx < l * k; idx += HM_THREADS) {
    int i = idx % l, jj = idx / l;
    Xs[idx] = Vrot[(int64_t)s.order[jj] * l + i];
  }
  cta_apply_q_rows<float>(J, l, l, l, s.tauB, Xs, l, k, s);
  for (int idx = tid; idx < gl * k; idx += HM_THREADS) {
    int i = idx % gl, jj = idx / gl;
    Ys[idx] = i < l ? Xs[i + (int64_t)jj * l] : 0.f;
  }
  cta_apply_q_rows<float>(stkM, gl, gl, l, tsM, Ys, gl, k, s);
  float* Cr = g.SAf;  // this member's rows of C (ld m), SA is no longer needed
  for (int idx = tid; idx < rm * k; idx += HM_THREADS) {
    int i = idx % rm, jj = idx / rm;
    Cr[(int64_t)jj * m + ra + i] = i < l ? Ys[(int64_t)r * l + i + (int64_t)jj * gl] : 0.f;
  }
  cta_apply_q_rows<float>(g.Mh + ra, m, rm, l, tauM, Cr + ra, m, k, s);
  // D: P W(:, order) S through the stack of SB and this member's block of SB
  for (int idx = tid; idx < l * k; idx += HM_THREADS) Xs[idx] = 0.f;
  __syncthreads();
  for (int idx = tid; idx < l * k; idx += HM_THREADS) {
    int j = idx % l, jj = idx / l;
    Xs[(int64_t)jj * l + perm[j]] = W[(int64_t)s.order[jj] * l + j];
  }
  __syncthreads();
  for (int idx = tid; idx < gl * k; idx += HM_THREADS) {
    int i = idx % gl, jj = idx / gl;
    Ys[idx] = i < l ? Xs[i + (int64_t)jj * l] : 0.f;
  }
  cta_apply_q_rows<float>(stkB, gl, gl, l, tsB, Ys, gl, k, s);
  for (int idx = tid; idx < rn * k; idx += HM_THREADS) {
    int i = idx % rn, jj = idx / rn;
    g.Vs[(int64_t)jj * n + ca + i] = i < l ? Ys[(int64_t)r * l + i + (int64_t)jj * gl] : 0.f;
  }
  cta_apply_q_rows<float>(g.SBf + ca, n, rn, l, tauB, g.Vs + ca, n, k, s);
  // 8. every member's rows finite?  Then the result, in FP64
  int bad = 0;
  for (int idx = tid; idx < rm * k; idx += HM_THREADS)
    if (!isfinite(Cr[(int64_t)(idx / rm) * m + ra + idx % rm])) bad = 1;
  for (int idx = tid; idx < rn * k; idx += HM_THREADS)
    if (!isfinite(g.Vs[(int64_t)(idx / rn) * n + ca + idx % rn])) bad = 1;
  bad = __syncthreads_or(bad);
  if (tid == 0) g.xch[(int64_t)r * HM_GANG_XCH + 6] = bad;
  gang_sync(e, c0, 4, G);
  bool anybad = false;
  for (int q = 0; q < G; ++q) anybad = anybad || g.xch[(int64_t)q * HM_GANG_XCH + 6] != 0.0;
  if (anybad) {
    gang_leave(e, c0, 4, 5);
    if (r == 0) gang_fallback(e, t, s, ti);  // the inputs are untouched so far
    return;
  }
  double* Uout = loc(e, t.e);
  double* Vout = loc(e, t.f);
  for (int idx = tid; idx < rm * k; idx += HM_THREADS) {
    int i = idx % rm, jj = idx / rm;
    Uout[(int64_t)jj * t.lde + ra + i] = (double)Cr[(int64_t)jj * m + ra + i];
  }
  for (int idx = tid; idx < rn * k; idx += HM_THREADS) {
    int i = idx % rn, jj = idx / rn;
    Vout[(int64_t)jj * t.ldf + ca + i] = (double)g.Vs[(int64_t)jj * n + ca + i] * S;
  }
  gang_sync(e, c0, 5, G);
  if (r == 0 && tid == 0) {
    if (s.ivals[13]) set_status(e.status, DS_RANK);
    if (t.rout >= 0) e.ranks[t.rout] = k;
    atomicAdd(e.counters, 1ull);
    atomicAdd(e.counters + 1, 1ull);
    atomicAdd(e.counters + 11, 1ull);  // truncations run by a gang
  }
  if (r == 0)
    count_f32(s, 2.0 * (n + m) * (double)l * l + (double)m * l * l + 4.0 * (double)G * l * l * l +
                     4.0 * (m + n) * (double)l * k);
}

__device__ void task_rkadd(const ExecEnv& e, const HTask& t, Smem& s, long long ti) {
  int m = t.m, n = t.n;
  bool aid = t.flags & F_A_IDENT, bid = t.flags & F_B_IDENT, btr = t.flags & F_B_TRANS;
  int w = aid ? m : (bid ? n : width_of(e, t.wa));
  int kin = t.rin >= 0 ? e.ranks[t.rin] : 0;
  const double* A = loc(e, t.a);
  const double* B = loc(e, t.b);
  const double* Uin = loc(e, t.c);
  const double* Vin = loc(e, t.d);
  double* Uout = loc(e, t.e);
  double* Vout = loc(e, t.f);
  bool zero = (w == 0);
  if (!zero && (t.flags & F_CHECK_ZERO)) {
    bool za = aid ? false : cta_all_zero(A, t.lda, m, w, s);
    bool zb = bid ? false : (btr ? cta_all_zero(B, t.ldb, w, n, s) : cta_all_zero(B, t.ldb, n, w, s));
    zero = za || zb;
  }
  if (zero) {
    if (Uout != Uin && kin > 0) {
      cta_copy(Uout, t.lde, Uin, t.ldc, m, kin, false, 1.0);
      cta_copy(Vout, t.ldf, Vin, t.ldd, n, kin, false, 1.0);
    }
    if (threadIdx.x == 0 && t.rout >= 0) e.ranks[t.rout] = kin;
    return;
  }
  int l = w + kin;
  if (l > HM_LMAX) {
    if (threadIdx.x == 0) set_status(e.status, DS_INTERNAL);
    return;
  }
  double* ws = loc(e, t.ws);
  double* SA = ws;
  double* SB = SA + (int64_t)m * l;
  double* W = SB + (int64_t)n * l;
  double* Jg = W + (int64_t)m * l;
  for (int idx = threadIdx.x; idx < m * l; idx += HM_THREADS) {
    int i = idx % m, j = idx / m;
    double v;
    if (j < w) v = t.alpha * (aid ? (i == j ? 1.0 : 0.0) : A[(int64_t)j * t.lda + i]);
    else v = Uin[(int64_t)(j - w) * t.ldc + i];
    SA[idx] = v;
  }
  for (int idx = threadIdx.x; idx < n * l; idx += HM_THREADS) {
    int i = idx % n, j = idx / n;
    double v;
    if (j < w) v = bid ? (i == j ? 1.0 : 0.0) : (btr ? B[(int64_t)i * t.ldb + j] : B[(int64_t)j * t.ldb + i]);
    else v = Vin[(int64_t)(j - w) * t.ldd + i];
    SB[idx] = v;
  }
  __syncthreads();
  double f = 0.0;
  // FP32 factored path (QR of the second factor) when l <= min(m, n); the
  // explicit FP32 path for the identity cases and the other small blocks
  bool fact = !aid && !bid && l <= m && l <= n;
  if (e.mixed && e.eps >= HM_F32_MIN_EPS && l >= e.rand_min_l && (!fact || l > HM_FACT32_DIRECT) &&
      (int64_t)m * n <= HM_F32_MAX_MN && (int64_t)m * n <= 4 * (int64_t)(m + n) * l) {
    // Mixed precision: M formed once (FP64 sums, FP32 copy), FP32 sketch and
    // projections, FP64 core.
    int Rr = m < n ? m : n;
    if (Rr > HM_RMAX) Rr = HM_RMAX;
    int64_t mn = (int64_t)m * n, fl = mn + 2 * (int64_t)(m + n) * Rr;
    float* gfw = (float*)(Jg + 2 * (int64_t)l * l);
    float* fw = fl <= HM_F32_SMEM ? (float*)s.jac : gfw;
    uint32_t* Om = (uint32_t*)(gfw + fl);
    float* Mf = fw;
    // M / S in FP32: base alpha Bhat^T or alpha Ahat (identity cases) plus the
    // stacked factors' products
    M32Part part;
    int j0 = (aid || bid) ? w : 0;
    part.SA = SA + (int64_t)j0 * m;
    part.SB = SB + (int64_t)j0 * n;
    part.k = l - j0;
    part.n = n;
    part.c0 = 0;
    auto base = [&](int i, int c) -> double {
      double v = aid ? (btr ? B[(int64_t)c * t.ldb + i] : B[(int64_t)i * t.ldb + c]) : A[(int64_t)c * t.lda + i];
      return t.alpha * v;
    };
    double mx = 0.0;
    int fs = form_m32(m, n, &part, 1, aid || bid, base, Mf, (float*)(Om + n), e.eps, &mx, s);
    if (fs == 1) record_bad(e, 9, m, n, l, kin, mx);
    int r0 = sketch_width(e, ti, kin, l, s);
    uint64_t seed = e.seed ^ ((uint64_t)blockIdx.x << 40) ^ (uint64_t)(t.rout + 1) * 0x9E3779B97F4A7C15ull;
    int ok = 0;
    int k = fs ? 0
               : trunc_rand32(Mf, m, n, mx, Mf + mn, Om, e.eps, t.cap, Uout, t.lde, Vout, t.ldf, e.status, s, &f,
                              &ok, seed, r0);
    if (ok && !cta_finite(Uout, t.lde, m, k, Vout, t.ldf, n)) {
      ok = 0;
      record_bad(e, 1, m, n, l, k, mx);
    }
    if (ok) {
      if (threadIdx.x == 0) {
        if (t.rout >= 0) e.ranks[t.rout] = k;
        atomicAdd(e.counters, 1ull);
        atomicAdd(e.counters + 1, 1ull);
        atomicAdd(e.flops, f);
      }
      count_sketch(e, s, ti, l, 1, k);
      return;
    }
    if (threadIdx.x == 0) atomicAdd(e.counters + 2, 1ull);
    count_sketch(e, s, ti, l, 0, 0);
  } else if (e.mixed && e.eps >= HM_F32_MIN_EPS && l >= e.rand_min_l && fact) {
    // factored M: FP32 steps of Fig. rkadd (randomised core only for l > 64)
    int r0 = sketch_width(e, ti, kin, l, s);
    uint64_t seed = e.seed ^ ((uint64_t)blockIdx.x << 40) ^ (uint64_t)(t.rout + 3) * 0x9E3779B97F4A7C15ull;
    int ok = 0;
    int k = task_fact32(e, t, s, m, n, l, SA, SB, n, l, nullptr, 0, 0, Jg + 2 * (int64_t)l * l, seed, r0, &f, &ok);
    if (ok) {
      if (threadIdx.x == 0) {
        if (t.rout >= 0) e.ranks[t.rout] = k;
        atomicAdd(e.counters, 1ull);
        atomicAdd(e.counters + 1, 1ull);
        atomicAdd(e.flops, f);
      }
      count_sketch(e, s, ti, l, 1, k);
      return;
    }
    if (threadIdx.x == 0) atomicAdd(e.counters + 2, 1ull);
    count_sketch(e, s, ti, l, 0, 0);
  } else if (e.mixed && e.eps > 0.0 && l >= e.rand_min_l) {
    // Randomised truncation; M explicit when that is the smaller form.
    double* R = Jg + 2 * (int64_t)l * l;
    const double* Md = nullptr;
    if ((int64_t)m * n <= (int64_t)(m + n) * l) {
      double* Mx = R;
      R += (int64_t)m * n;
      for (int idx = threadIdx.x; idx < m * n; idx += HM_THREADS) {
        int i = idx % m, c = idx / m;
        double v;
        if (aid) v = btr ? B[(int64_t)c * t.ldb + i] : B[(int64_t)i * t.ldb + c];   // alpha Bhat^T
        else if (bid) v = A[(int64_t)c * t.lda + i];                                // alpha Ahat
        else {
          v = 0.0;
          for (int j = 0; j < w; ++j)
            v += A[(int64_t)j * t.lda + i] * (btr ? B[(int64_t)c * t.ldb + j] : B[(int64_t)j * t.ldb + c]);
        }
        v *= t.alpha;
        for (int j = 0; j < kin; ++j) v += Uin[(int64_t)j * t.ldc + i] * Vin[(int64_t)j * t.ldd + c];
        Mx[idx] = v;
      }
      __syncthreads();
      Md = Mx;
      f += 2.0 * m * n * (double)(kin + ((aid || bid) ? 0 : w));
    }
    RandIn ri;
    ri.m = m;
    ri.n = n;
    ri.l = l;
    ri.Md = Md;
    ri.SA = SA;
    ri.SB = SB;
    ri.ws = R;
    ri.seed = e.seed ^ ((uint64_t)blockIdx.x << 40) ^ (uint64_t)(t.rout + 1) * 0x9E3779B97F4A7C15ull;
    ri.r0 = sketch_width(e, ti, kin, l, s);
    int ok = 0;
    int k = trunc_rand(ri, e.eps, t.cap, Uout, t.lde, Vout, t.ldf, e.status, s, &f, &ok);
    if (ok) {
      if (threadIdx.x == 0) {
        if (t.rout >= 0) e.ranks[t.rout] = k;
        atomicAdd(e.counters, 1ull);
        atomicAdd(e.counters + 1, 1ull);
        atomicAdd(e.flops, f);
      }
      count_sketch(e, s, ti, l, 2, k);
      return;
    }
    if (threadIdx.x == 0) atomicAdd(e.counters + 2, 1ull);
    count_sketch(e, s, ti, l, 0, 0);
  }
  TruncIn in;
  in.nb = 1;
  in.m = m;
  in.n[0] = n;
  in.k[0] = l;
  in.SA[0] = SA;
  in.SB[0] = SB;
  in.W = W;
  in.Jg = Jg;
  int k = trunc_core(in, e.eps, t.cap, Uout, t.lde, Vout, t.ldf, e.status, s, &f, e.rank_rule);
  if (threadIdx.x == 0) {
    if (t.rout >= 0) e.ranks[t.rout] = k;
    atomicAdd(e.counters, 1ull);
    atomicAdd(e.flops, f);
  }
  record_rank(e, ti, l, k);
  note_exact(e, ti, l, k);
}

__device__ void task_rowmerge(const ExecEnv& e, const HTask& t, Smem& s, long long ti) {
  int m = t.m;
  int n0 = t.p, n1 = t.q;
  int k0 = width_of(e, t.wa), k1 = width_of(e, t.wb);
  double* Uout = loc(e, t.e);
  double* Vout = loc(e, t.f);
  if (k0 + k1 > HM_LMAX) {
    if (threadIdx.x == 0) set_status(e.status, DS_INTERNAL);
    return;
  }
  if (k0 + k1 == 0) {
    if (threadIdx.x == 0 && t.rout >= 0) e.ranks[t.rout] = 0;
    return;
  }
  double* ws = loc(e, t.ws);
  double* SA0 = ws;
  double* SA1 = SA0 + (int64_t)m * k0;
  double* SB0 = SA1 + (int64_t)m * k1;
  double* SB1 = SB0 + (int64_t)n0 * k0;
  double* W = SB1 + (int64_t)n1 * k1;
  double* Jg = W + (int64_t)m * (k0 + k1);
  cta_copy(SA0, m, loc(e, t.a), t.lda, m, k0, false, 1.0);
  cta_copy(SB0, n0, loc(e, t.b), t.ldb, n0, k0, false, 1.0);
  cta_copy(SA1, m, loc(e, t.c), t.ldc, m, k1, false, 1.0);
  cta_copy(SB1, n1, loc(e, t.d), t.ldd, n1, k1, false, 1.0);
  __syncthreads();
  double f = 0.0;
  int l = k0 + k1;
  int n = n0 + n1;
  bool fact = l <= m && l <= n;
  if (e.mixed && e.eps >= HM_F32_MIN_EPS && l >= e.rand_min_l && (!fact || l > HM_FACT32_DIRECT) &&
      (int64_t)m * n <= HM_F32_MAX_MN && (int64_t)m * n <= 4 * (int64_t)(m + n) * l) {
    int Rr = m < n ? m : n;
    if (Rr > HM_RMAX) Rr = HM_RMAX;
    int64_t mn = (int64_t)m * n, fl = mn + 2 * (int64_t)(m + n) * Rr;
    float* gfw = (float*)(Jg + 2 * (int64_t)l * l);
    float* fw = fl <= HM_F32_SMEM ? (float*)s.jac : gfw;
    uint32_t* Om = (uint32_t*)(gfw + fl);
    float* Mf = fw;
    M32Part parts[2];
    parts[0].SA = SA0;
    parts[0].SB = SB0;
    parts[0].k = k0;
    parts[0].n = n0;
    parts[0].c0 = 0;
    parts[1].SA = SA1;
    parts[1].SB = SB1;
    parts[1].k = k1;
    parts[1].n = n1;
    parts[1].c0 = n0;
    auto nobase = [](int, int) -> double { return 0.0; };
    double mx = 0.0;
    int fs = form_m32(m, n, parts, 2, false, nobase, Mf, (float*)(Om + n), e.eps, &mx, s);
    if (fs == 1) record_bad(e, 10, m, n, l, k0, mx);
    int r0 = sketch_width(e, ti, k0 > k1 ? k0 : k1, l, s);
    uint64_t seed = e.seed ^ ((uint64_t)blockIdx.x << 40) ^ (uint64_t)(t.rout + 7) * 0x9E3779B97F4A7C15ull;
    int ok = 0;
    int k = fs ? 0
               : trunc_rand32(Mf, m, n, mx, Mf + mn, Om, e.eps, t.cap, Uout, t.lde, Vout, t.ldf, e.status, s, &f,
                              &ok, seed, r0);
    if (ok && !cta_finite(Uout, t.lde, m, k, Vout, t.ldf, n)) {
      ok = 0;
      record_bad(e, 2, m, n, l, k, mx);
    }
    if (ok) {
      if (threadIdx.x == 0) {
        if (t.rout >= 0) e.ranks[t.rout] = k;
        atomicAdd(e.counters, 1ull);
        atomicAdd(e.counters + 1, 1ull);
        atomicAdd(e.flops, f);
      }
      count_sketch(e, s, ti, l, 1, k);
      return;
    }
    if (threadIdx.x == 0) atomicAdd(e.counters + 2, 1ull);
    count_sketch(e, s, ti, l, 0, 0);
  } else if (e.mixed && e.eps >= HM_F32_MIN_EPS && l >= e.rand_min_l && fact) {
    // [A_0 A_1] blockdiag(B_0, B_1)^T: FP32 steps of Fig. rkadd
    int r0 = sketch_width(e, ti, k0 > k1 ? k0 : k1, l, s);
    uint64_t seed = e.seed ^ ((uint64_t)blockIdx.x << 40) ^ (uint64_t)(t.rout + 5) * 0x9E3779B97F4A7C15ull;
    int ok = 0;
    int k = task_fact32(e, t, s, m, n, l, SA0, SB0, n0, k0, SB1, n1, k1, Jg + 2 * (int64_t)l * l, seed, r0, &f, &ok);
    if (ok) {
      if (threadIdx.x == 0) {
        if (t.rout >= 0) e.ranks[t.rout] = k;
        atomicAdd(e.counters, 1ull);
        atomicAdd(e.counters + 1, 1ull);
        atomicAdd(e.flops, f);
      }
      count_sketch(e, s, ti, l, 1, k);
      return;
    }
    if (threadIdx.x == 0) atomicAdd(e.counters + 2, 1ull);
    count_sketch(e, s, ti, l, 0, 0);
  } else if (e.mixed && e.eps > 0.0 && l >= e.rand_min_l) {
    // [A_0 A_1] blockdiag(B_0, B_1)^T with SA = [SA0 SA1] (contiguous)
    double* SBd = Jg + 2 * (int64_t)l * l;
    double* R = SBd + (int64_t)n * l;
    for (int idx = threadIdx.x; idx < n * l; idx += HM_THREADS) {
      int i = idx % n, j = idx / n;
      double v = 0.0;
      if (j < k0 && i < n0) v = SB0[(int64_t)j * n0 + i];
      else if (j >= k0 && i >= n0) v = SB1[(int64_t)(j - k0) * n1 + (i - n0)];
      SBd[idx] = v;
    }
    __syncthreads();
    const double* Md = nullptr;
    if ((int64_t)m * n <= (int64_t)(m + n) * l) {
      double* Mx = R;
      R += (int64_t)m * n;
      for (int idx = threadIdx.x; idx < m * n; idx += HM_THREADS) {
        int i = idx % m, c = idx / m;
        double v = 0.0;
        if (c < n0) {
          for (int j = 0; j < k0; ++j) v += SA0[(int64_t)j * m + i] * SB0[(int64_t)j * n0 + c];
        } else {
          for (int j = 0; j < k1; ++j) v += SA1[(int64_t)j * m + i] * SB1[(int64_t)j * n1 + (c - n0)];
        }
        Mx[idx] = v;
      }
      __syncthreads();
      Md = Mx;
      f += 2.0 * m * (double)(n0 * k0 + n1 * k1);
    }
    RandIn ri;
    ri.m = m;
    ri.n = n;
    ri.l = l;
    ri.Md = Md;
    ri.SA = SA0;
    ri.SB = SBd;
    ri.ws = R;
    ri.seed = e.seed ^ ((uint64_t)blockIdx.x << 40) ^ (uint64_t)(t.rout + 7) * 0x9E3779B97F4A7C15ull;
    ri.r0 = sketch_width(e, ti, k0 > k1 ? k0 : k1, l, s);
    int ok = 0;
    int k = trunc_rand(ri, e.eps, t.cap, Uout, t.lde, Vout, t.ldf, e.status, s, &f, &ok);
    if (ok) {
      if (threadIdx.x == 0) {
        if (t.rout >= 0) e.ranks[t.rout] = k;
        atomicAdd(e.counters, 1ull);
        atomicAdd(e.counters + 1, 1ull);
        atomicAdd(e.flops, f);
      }
      count_sketch(e, s, ti, l, 2, k);
      return;
    }
    if (threadIdx.x == 0) atomicAdd(e.counters + 2, 1ull);
    count_sketch(e, s, ti, l, 0, 0);
  }
  TruncIn in;
  in.nb = 2;
  in.m = m;
  in.n[0] = n0;
  in.n[1] = n1;
  in.k[0] = k0;
  in.k[1] = k1;
  in.SA[0] = SA0;
  in.SA[1] = SA1;
  in.SB[0] = SB0;
  in.SB[1] = SB1;
  in.W = W;
  in.Jg = Jg;
  int k = trunc_core(in, e.eps, t.cap, Uout, t.lde, Vout, t.ldf, e.status, s, &f, e.rank_rule);
  if (threadIdx.x == 0) {
    if (t.rout >= 0) e.ranks[t.rout] = k;
    atomicAdd(e.counters, 1ull);
    atomicAdd(e.flops, f);
  }
  record_rank(e, ti, l, k);
  note_exact(e, ti, l, k);
}

// FP64 operations of the non-truncation tasks: this lane's share (warp 0
// sums the shares; leaf lists are split over the lanes, everything else is
// lane 0's).
__device__ double task_flops(const ExecEnv& e, const HTask& t, int lane) {
  if (lane != 0 && t.type != T_HMV && t.type != T_DENSIFY) return 0.0;
  switch (t.type) {
    case T_LU:
      return 2.0 / 3.0 * (double)t.m * t.m * t.m;
    case T_TRSM:
      return (double)t.m * t.m * width_of(e, t.wa);
    case T_INV:
      return 2.0 * t.m * (double)t.m * t.m;
    case T_CHOL:
      return (double)t.m * t.m * t.m / 3.0;
    case T_GEMM:
      return 2.0 * t.m * t.n * (double)width_of(e, t.wa);
    case T_ADD:
      return (double)t.m * t.n;
    case T_HMV: {
      double w = width_of(e, t.wa), f = 0.0;
      for (int li = lane; li < t.list_len; li += 32) {
        const LeafRef& L = e.leaves[t.list_begin + li];
        if (L.kind == 1) f += 2.0 * L.rows * L.cols * w;
        else f += 2.0 * e.ranks[L.rank_slot] * (double)(L.rows + L.cols) * w;
      }
      return f;
    }
    case T_DENSIFY: {
      double f = 0.0;
      for (int li = lane; li < t.list_len; li += 32) {
        const LeafRef& L = e.leaves[t.list_begin + li];
        if (L.kind == 2) f += 2.0 * e.ranks[L.rank_slot] * (double)L.rows * L.cols;
      }
      return f;
    }
    default:
      return 0.0;
  }
}

// Algorithmic bytes of a task: what it must read and write once (FP64),
// e.g. 8 [(m + n) l + (m + n) k] for a truncation of stacked width l to rank
// k; l_in is the stacked width read before the task ran (-1: not a
// truncation).  This lane's share, as in task_flops.
__device__ double task_bytes(const ExecEnv& e, const HTask& t, int l_in, int lane) {
  if (lane != 0 && t.type != T_HMV && t.type != T_DENSIFY) return 0.0;
  switch (t.type) {
    case T_LU:
    case T_INV:
    case T_CHOL:
      return 16.0 * t.m * t.m;
    case T_TRSM:
      return 8.0 * ((double)t.m * t.m + 2.0 * t.m * width_of(e, t.wa));
    case T_GEMM: {
      double w = width_of(e, t.wa);
      return 8.0 * (2.0 * t.m * t.n + (t.m + t.n) * w);
    }
    case T_ADD:
      return 24.0 * t.m * t.n;
    case T_COPY:
      return 16.0 * t.m * t.n;
    case T_ZERO:
      return 8.0 * t.m * t.n;
    case T_HMV:
    case T_DENSIFY: {
      double w = t.type == T_HMV ? width_of(e, t.wa) : 0.0, b = 0.0;
      for (int li = lane; li < t.list_len; li += 32) {
        const LeafRef& L = e.leaves[t.list_begin + li];
        double f = L.kind == 1 ? (double)L.rows * L.cols : (double)e.ranks[L.rank_slot] * (L.rows + L.cols);
        b += 8.0 * (f + (t.type == T_HMV ? 2.0 * (L.rows + L.cols) * w : (double)L.rows * L.cols));
      }
      return b;
    }
    case T_RKADD:
    case T_ROWMERGE: {
      // a gang's bytes are counted once, by member 0
      if (l_in <= 0 || (t.pad1 > 1 && t.pad0 != 0)) return 0.0;
      int n = (t.type == T_RKADD || t.pad1 > 1) ? t.n : t.p + t.q;
      int k = t.rout >= 0 ? e.ranks[t.rout] : 0;
      return 8.0 * ((double)(t.m + n) * l_in + (double)(t.m + n) * k);
    }
    default:
      return 0.0;
  }
}

// Stacked width of a truncation task before it runs (rank slots are
// overwritten in place).
__device__ int trunc_width(const ExecEnv& e, const HTask& t) {
  if (t.type == T_RKADD) {
    bool aid = t.flags & F_A_IDENT, bid = t.flags & F_B_IDENT;
    int w = aid ? t.m : (bid ? t.n : width_of(e, t.wa));
    return w + (t.rin >= 0 ? e.ranks[t.rin] : 0);
  }
  if (t.type == T_ROWMERGE) return width_of(e, t.wa) + width_of(e, t.wb);
  return -1;
}

__device__ void run_task(const ExecEnv& e, const HTask& t, Smem& s, long long ti) {
  // FP32 leaf products and solves in the mixed path (eps >= HM_F32_MIN_EPS)
  bool f32 = e.mixed && e.eps >= HM_F32_MIN_EPS;
  switch (t.type) {
    case T_NOP:
      break;
    case T_LU:
      cta_lu(loc(e, t.a), t.lda, t.m, e.status);
      break;
    case T_TRSM:
      if (!(f32 && cta_trsm_f32(t.p, loc(e, t.a), t.lda, t.m, loc(e, t.b), t.ldb, width_of(e, t.wa), s)))
        cta_trsm(t.p, loc(e, t.a), t.lda, t.m, loc(e, t.b), t.ldb, width_of(e, t.wa), s);
      break;
    case T_HMV:
      task_hmv(e, t, s, f32);
      if (t.pad1 > 1) {
        // a gang of H x thin-dense products on disjoint output rows: member 0
        // finishes (and releases the successors) after every member
        if (t.pad0 == 0) gang_sync(e, ti, 1, t.pad1);
        else gang_leave(e, ti - t.pad0, 0, 1);
      }
      break;
    case T_DENSIFY:
      task_densify(e, t, s);
      break;
    case T_GEMM: {
      int w = width_of(e, t.wa);
      bool zero = t.flags & F_ZERO_OUT;
      if (f32 && (w > 0 || zero)) {
        cta_gemm32(loc(e, t.c), t.ldc, t.m, t.n, w, t.alpha, loc(e, t.a), t.lda, false, loc(e, t.b), t.ldb,
                   !(t.flags & F_B_TRANS), zero, (float*)s.jac);
        count_f32(s, 2.0 * t.m * (double)t.n * w);
      }
      else if (w > 0 || zero)
        cta_gemm(loc(e, t.c), t.ldc, t.m, t.n, w, t.alpha, loc(e, t.a), t.lda, false, loc(e, t.b), t.ldb,
                 !(t.flags & F_B_TRANS), zero);
      break;
    }
    case T_ADD: {
      double* C = loc(e, t.c);
      const double* A = loc(e, t.a);
      bool tr = t.flags & F_TRANS;
      for (int idx = threadIdx.x; idx < t.m * t.n; idx += HM_THREADS) {
        int i = idx % t.m, j = idx / t.m;
        C[(int64_t)j * t.ldc + i] += t.alpha * (tr ? A[(int64_t)i * t.lda + j] : A[(int64_t)j * t.lda + i]);
      }
      break;
    }
    case T_COPY:
      cta_copy(loc(e, t.c), t.ldc, loc(e, t.a), t.lda, t.m, t.n, t.flags & F_TRANS, 1.0);
      break;
    case T_ZERO: {
      double* C = loc(e, t.c);
      for (int idx = threadIdx.x; idx < t.m * t.n; idx += HM_THREADS) C[(int64_t)(idx / t.m) * t.ldc + idx % t.m] = 0.0;
      break;
    }
    case T_RANKSET:
      if (threadIdx.x == 0) e.ranks[t.rout] = width_of(e, t.wa);
      break;
    case T_INV:
      task_inv(e, t, s);
      break;
    case T_CHOL:
      task_chol(e, t, s);
      break;
    case T_RKADD:
      if (t.pad1 > 1) task_rkadd_gang(e, t, s, ti);
      else task_rkadd(e, t, s, ti);
      break;
    case T_ROWMERGE:
      if (t.pad1 > 1) task_rkadd_gang(e, t, s, ti);
      else task_rowmerge(e, t, s, ti);
      break;
    default:
      if (threadIdx.x == 0) set_status(e.status, DS_INTERNAL);
  }
}

__global__ void __launch_bounds__(HM_THREADS, 1) exec_tasks(ExecEnv e) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem& s = *reinterpret_cast<Smem*>(smem_raw);
  __shared__ long long cur;
  __shared__ int skip;
  __shared__ uint64_t cur_t0;
  for (;;) {
    if (threadIdx.x == 0) {
      cur = (long long)atomicAdd(e.head, 1ull);
      skip = 0;
      if (cur < e.ntasks) {
        // bounded wait on every predecessor
        int64_t d0 = e.dep_ptr[cur], d1 = e.dep_ptr[cur + 1];
        uint64_t t0 = global_ns();
        s.ivals[8] = (int)(t0 & 0x7fffffff);
        for (int64_t d = d0; d < d1 && !skip; ++d) {
          const int* flag = e.done + e.dep_idx[d];
          int64_t it = 0;
          while (ld_acquire(flag) == 0) {
            if (++it > e.spin_iters || global_ns() - t0 > e.spin_ns) {
              set_status(e.status, DS_TIMEOUT);
              skip = 1;
              break;
            }
            __nanosleep(64);
          }
        }
        if (ld_acquire(e.status) != 0) skip = 1;
        hm_status_won = 0;
        uint64_t t1 = global_ns();
        atomicAdd(e.wait_ns, (unsigned long long)(t1 - t0));
        cur_t0 = t1;
      }
    }
    __syncthreads();
    long long t = cur;
    if (t >= e.ntasks) break;
    if (!skip) {
      HTask task = e.tasks[t];
      if (threadIdx.x == 0) s.bcast[7] = 0.0;
      int l_in = 0;
      if (threadIdx.x == 0) l_in = trunc_width(e, task);
      __syncthreads();  // every thread has read the rank slots the task may overwrite
      run_task(e, task, s, t);
      __syncthreads();
      if (threadIdx.x == 0 && hm_status_won) *e.fail_task = t + 1;
      if (threadIdx.x < 32) {
        // the task's counts (a task changes no rank that its own count reads)
        l_in = __shfl_sync(0xffffffffu, l_in, 0);
        double b = warp_sum(task_bytes(e, task, l_in, threadIdx.x));
        double f = (task.type != T_RKADD && task.type != T_ROWMERGE) ? warp_sum(task_flops(e, task, threadIdx.x))
                                                                       : 0.0;
        if (threadIdx.x == 0 && b > 0.0) atomicAdd(e.bytes, b);
        if (threadIdx.x == 0 && f > 0.0) atomicAdd(e.flops, f);
      }
      if (threadIdx.x == 0 && s.bcast[7] > 0.0) atomicAdd(e.flops32, s.bcast[7]);
      if (threadIdx.x == 0 && task.type >= 0 && task.type < 16) {
        uint64_t dt = global_ns() - cur_t0;
        atomicAdd(e.type_ns + task.type, (unsigned long long)dt);
        atomicAdd(e.type_cnt + task.type, 1ull);
        if (e.task_ns) e.task_ns[t] = (uint32_t)(dt < 0xffffffffull ? dt : 0xffffffffull);
      }
    }
    if (skip && threadIdx.x == 0) {
      // a skipped gang member still arrives at all its gang's barriers
      const HTask& sk = e.tasks[t];
      if ((sk.type == T_RKADD || sk.type == T_ROWMERGE || sk.type == T_HMV) && sk.pad1 > 1)
        atomicAdd(e.gang + (t - sk.pad0), sk.type == T_HMV ? 1 : 5);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      st_release(e.done + t, 1);
    }
  }
}

// ---------------------------------------------------------------------------
// Batched truncation of independent low-rank matrices in place.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(HM_THREADS) trunc_batched(const TruncProblem* probs, double eps, int* status,
                                                           int mixed) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem& s = *reinterpret_cast<Smem*>(smem_raw);
  const TruncProblem P = probs[blockIdx.x];
  int m = P.m, n = P.n, l = P.k;
  if (l > HM_LMAX) {
    if (threadIdx.x == 0) set_status(status, DS_INTERNAL);
    return;
  }
  double* SA = P.ws;
  double* SB = SA + (int64_t)m * l;
  double* W = SB + (int64_t)n * l;
  double* Jg = W + (int64_t)m * l;
  cta_copy(SA, m, P.U, P.ldu, m, l, false, 1.0);
  cta_copy(SB, n, P.V, P.ldv, n, l, false, 1.0);
  __syncthreads();
  int cap = l < m ? l : m;
  if (n < cap) cap = n;
  if (mixed && eps >= HM_F32_MIN_EPS && l > 0 && l <= m && l <= n && l <= HM_FACT32_DIRECT) {
    // factored stack: the FP32 steps of Fig. rkadd, no sketch (as hmat_lu's mixed form)
    int ok = 0;
    double S = 0.0, f = 0.0;
    int k = fact32_run(m, n, l, SA, SB, n, l, nullptr, 0, 0, Jg + 2 * (int64_t)l * l, eps, cap, P.U, P.ldu, P.V, P.ldv,
                       status, s, 0x5EEDull + blockIdx.x, l, &f, &ok, &S);
    if (ok && cta_finite(P.U, P.ldu, m, k, P.V, P.ldv, n)) {
      if (threadIdx.x == 0) {
        P.k_new[0] = k;
        atomicAdd(status + 1, 1);
      }
      return;
    }
  } else if (mixed && eps >= HM_F32_MIN_EPS && (int64_t)m * n <= HM_F32_MAX_MN && l > 0) {
    int Rr = m < n ? m : n;
    if (Rr > HM_RMAX) Rr = HM_RMAX;
    int64_t mn = (int64_t)m * n, fl = mn + 2 * (int64_t)(m + n) * Rr;
    float* gfw = (float*)(Jg + 2 * (int64_t)l * l);
    float* Mf = fl <= HM_F32_SMEM ? (float*)s.jac : gfw;
    uint32_t* Om = (uint32_t*)(gfw + fl);
    auto entry = [&](int idx) {
      int i = idx % m, c = idx / m;
      double v = 0.0;
      for (int j = 0; j < l; ++j) v += SA[(int64_t)j * m + i] * SB[(int64_t)j * n + c];
      return v;
    };
    double mx = 0.0;
    for (int idx = threadIdx.x; idx < mn; idx += HM_THREADS) mx = fmax(mx, fabs(entry(idx)));
    mx = block_max(mx, s);
    double inv = mx > 0.0 ? 1.0 / mx : 0.0;
    for (int idx = threadIdx.x; idx < mn; idx += HM_THREADS) Mf[idx] = (float)(entry(idx) * inv);
    __syncthreads();
    int ok = 0;
    int k = trunc_rand32(Mf, m, n, mx, Mf + mn, Om, eps, cap, P.U, P.ldu, P.V, P.ldv, status, s, nullptr, &ok,
                         0x5EEDull + blockIdx.x, 8);
    if (ok) {
      if (threadIdx.x == 0) {
        P.k_new[0] = k;
        atomicAdd(status + 1, 1);
      }
      return;
    }
  }
  TruncIn in;
  in.nb = 1;
  in.m = m;
  in.n[0] = n;
  in.k[0] = l;
  in.SA[0] = SA;
  in.SB[0] = SB;
  in.W = W;
  in.Jg = Jg;
  int k = trunc_core(in, eps, cap, P.U, P.ldu, P.V, P.ldv, status, s);
  if (threadIdx.x == 0) P.k_new[0] = k;
}

// ---------------------------------------------------------------------------
// Construction from CSR (original ordering) and dense export.
// ---------------------------------------------------------------------------
__global__ void csr_scatter(const DenseLeafDesc* leaves, int nleaves, const int64_t* rowptr, const int64_t* colidx,
                            const double* val, const int64_t* perm, const int64_t* iperm, double* hbase,
                            unsigned long long* placed) {
  int b = blockIdx.x;
  if (b >= nleaves) return;
  DenseLeafDesc L = leaves[b];
  unsigned long long cnt = 0, bad = 0;
  for (int i = threadIdx.x; i < L.rows; i += blockDim.x) {
    int64_t p = perm[L.roff + i];
    for (int64_t e = rowptr[p]; e < rowptr[p + 1]; ++e) {
      int64_t j = iperm[colidx[e]] - L.coff;
      if (j >= 0 && j < L.cols) {
        double v = val[e];
        hbase[L.off + i + j * (int64_t)L.rows] += v;
        ++cnt;
        if (!isfinite(v)) ++bad;
      }
    }
  }
  if (cnt) atomicAdd(placed, cnt);
  if (bad) atomicAdd(placed + 1, bad);
}

__global__ void to_dense_kernel(const LeafRef* leaves, int nleaves, const double* hbase, const int* ranks,
                                double* out, int64_t ldo) {
  int b = blockIdx.x;
  if (b >= nleaves) return;
  LeafRef L = leaves[b];
  for (int idx = threadIdx.x; idx < L.rows * L.cols; idx += blockDim.x) {
    int i = idx % L.rows, j = idx / L.rows;
    double v = 0.0;
    if (L.kind == 1) {
      v = hbase[L.a + i + (int64_t)j * L.lda];
    } else {
      int k = ranks[L.rank_slot];
      for (int l = 0; l < k; ++l) v += hbase[L.a + i + (int64_t)l * L.lda] * hbase[L.b + j + (int64_t)l * L.ldb];
    }
    out[(L.roff + i) + (int64_t)(L.coff + j) * ldo] = v;
  }
}

// ---------------------------------------------------------------------------
// Conjugate-gradient building blocks (grid-stride loops over n x nrhs).
// ---------------------------------------------------------------------------
__global__ void permute_kernel(const double* src, double* dst, const int64_t* perm, int64_t n, int64_t nrhs,
                               int gather) {
  int64_t total = n * nrhs;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = idx % n, c = idx / n;
    if (gather) dst[idx] = src[c * n + perm[i]];
    else dst[c * n + perm[i]] = src[idx];
  }
}

// one warp per row, all right-hand sides of that row
__global__ void csr_spmv_kernel(int64_t n, const int64_t* rowptr, const int64_t* colidx, const double* val,
                                const double* X, double* Y, int64_t nrhs) {
  int lane = threadIdx.x & 31;
  int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
    int64_t e0 = rowptr[i], e1 = rowptr[i + 1];
    for (int64_t c = 0; c < nrhs; ++c) {
      double a = 0.0;
      for (int64_t e = e0 + lane; e < e1; e += 32) a += val[e] * X[c * n + colidx[e]];
      a = warp_sum(a);
      if (lane == 0) Y[c * n + i] = a;
    }
  }
}

// one block per column
__global__ void col_dots_kernel(int64_t n, const double* X, const double* Y, double* out) {
  __shared__ double red[32];
  int64_t c = blockIdx.x;
  double a = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) a += X[c * n + i] * Y[c * n + i];
  a = warp_sum(a);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x < 32) {
    double b = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    b = warp_sum(b);
    if (threadIdx.x == 0) out[c] = b;
  }
}

__global__ void cg_xr_kernel(int64_t n, int64_t nrhs, const double* alpha, const double* P, const double* Q,
                             double* X, double* R) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n * nrhs; idx += (int64_t)gridDim.x * blockDim.x) {
    double a = alpha[idx / n];
    X[idx] += a * P[idx];
    R[idx] -= a * Q[idx];
  }
}

__global__ void cg_p_kernel(int64_t n, int64_t nrhs, const double* beta, const double* Z, double* P) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n * nrhs; idx += (int64_t)gridDim.x * blockDim.x)
    P[idx] = Z[idx] + beta[idx / n] * P[idx];
}

__global__ void sub_kernel(int64_t count, const double* A, const double* B, double* D) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < count; idx += (int64_t)gridDim.x * blockDim.x)
    D[idx] = A[idx] - B[idx];
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
static int grid_for(int64_t work) {
  int64_t g = (work + 255) / 256;
  return (int)(g < 1 ? 1 : (g > 152 * 32 ? 152 * 32 : g));
}

cudaError_t launch_permute(const double* src, double* dst, const int64_t* perm, int64_t n, int64_t nrhs, bool gather,
                           cudaStream_t st) {
  (void)cudaGetLastError();
  permute_kernel<<<grid_for(n * nrhs), 256, 0, st>>>(src, dst, perm, n, nrhs, gather ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_csr_spmv(int64_t n, const int64_t* rowptr, const int64_t* colidx, const double* val,
                            const double* X, double* Y, int64_t nrhs, cudaStream_t st) {
  (void)cudaGetLastError();
  csr_spmv_kernel<<<grid_for(32 * n), 256, 0, st>>>(n, rowptr, colidx, val, X, Y, nrhs);
  return cudaGetLastError();
}

cudaError_t launch_col_dots(int64_t n, int64_t nrhs, const double* X, const double* Y, double* out, cudaStream_t st) {
  (void)cudaGetLastError();
  col_dots_kernel<<<(unsigned)nrhs, 1024, 0, st>>>(n, X, Y, out);
  return cudaGetLastError();
}

cudaError_t launch_cg_xr(int64_t n, int64_t nrhs, const double* alpha, const double* P, const double* Q, double* X,
                         double* R, cudaStream_t st) {
  (void)cudaGetLastError();
  cg_xr_kernel<<<grid_for(n * nrhs), 256, 0, st>>>(n, nrhs, alpha, P, Q, X, R);
  return cudaGetLastError();
}

cudaError_t launch_cg_p(int64_t n, int64_t nrhs, const double* beta, const double* Z, double* P, cudaStream_t st) {
  (void)cudaGetLastError();
  cg_p_kernel<<<grid_for(n * nrhs), 256, 0, st>>>(n, nrhs, beta, Z, P);
  return cudaGetLastError();
}

cudaError_t launch_sub(int64_t count, const double* A, const double* B, double* D, cudaStream_t st) {
  (void)cudaGetLastError();
  sub_kernel<<<grid_for(count), 256, 0, st>>>(count, A, B, D);
  return cudaGetLastError();
}
size_t smem_bytes() { return sizeof(Smem); }

cudaError_t launch_exec(const ExecEnv& env, int grid, cudaStream_t st) {
  (void)cudaGetLastError();  // a stale error of an earlier call is not this launch's
  exec_tasks<<<grid, HM_THREADS, sizeof(Smem), st>>>(env);
  return cudaGetLastError();
}

cudaError_t exec_occupancy(int* blocks_per_sm) {
  cudaError_t e = cudaFuncSetAttribute(exec_tasks, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem));
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, exec_tasks, HM_THREADS, sizeof(Smem));
}

cudaError_t launch_trunc_batched(const TruncProblem* probs, int count, double eps, int* status, int mixed,
                                 cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(trunc_batched, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem));
  if (e != cudaSuccess) return e;
  (void)cudaGetLastError();
  trunc_batched<<<count, HM_THREADS, sizeof(Smem), st>>>(probs, eps, status, mixed);
  return cudaGetLastError();
}

cudaError_t launch_csr_scatter(const DenseLeafDesc* leaves, int nleaves, const int64_t* rowptr, const int64_t* colidx,
                               const double* val, const int64_t* perm, const int64_t* iperm, double* hbase,
                               unsigned long long* placed, cudaStream_t st) {
  if (nleaves == 0) return cudaSuccess;
  (void)cudaGetLastError();
  csr_scatter<<<nleaves, 128, 0, st>>>(leaves, nleaves, rowptr, colidx, val, perm, iperm, hbase, placed);
  return cudaGetLastError();
}

cudaError_t launch_to_dense(const LeafRef* leaves, int nleaves, const double* hbase, const int* ranks, double* out,
                            int64_t ldo, cudaStream_t st) {
  if (nleaves == 0) return cudaSuccess;
  (void)cudaGetLastError();
  to_dense_kernel<<<nleaves, 256, 0, st>>>(leaves, nleaves, hbase, ranks, out, ldo);
  return cudaGetLastError();
}

}  // namespace hm
