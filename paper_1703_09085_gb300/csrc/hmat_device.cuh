// hmat_device.cuh -- CTA-level FP64 building blocks of the H-matrix tasks.
//
// Every routine here is executed by all HM_THREADS threads of one CTA and
// synchronises the CTA with __syncthreads(); none of them waits on another CTA.
// Matrices are column-major FP64 in global memory (L2 resident for the block
// sizes of the hot path); small square cores live in shared memory.
//
// Dense building blocks follow the textbook mathematics: Householder QR with
// reflectors P = I - tau v v^T, v = x - alpha e_j (Golub and Van Loan,
// Alg. 5.1.1; the column is scaled by its largest entry first where its
// squares would leave the floating-point range), row-parallel over the CTA;
// one-sided Jacobi SVD (Hestenes 1958; Demmel and Veselic 1992) with the
// parallel round-robin ordering; no-pivot Gaussian elimination.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "hmat_tasks.h"

#define HM_THREADS 256
#define HM_WARPS (HM_THREADS / 32)
#define HM_LMAX 256            // largest stacked width of a truncation
#ifndef HM_JAC_SMEM
#define HM_JAC_SMEM 9216       // doubles of shared memory for the cores and staged panels
#endif

namespace hm {

// Shared-memory layout of one CTA (dynamic shared memory).
struct Smem {
  double red[HM_WARPS * 2];
  double bcast[8];
  double tauB[HM_LMAX];
  double rdiagB[HM_LMAX];
  double tauA[HM_LMAX];
  double rdiagA[HM_LMAX];
  double sigma[HM_LMAX];
  int order[HM_LMAX];
  int ivals[16];
  // per-warp partial sums of the row-parallel FP32 factorisations (two
  // buffers, used alternately so that one barrier per step suffices)
  double redd[2][HM_WARPS * HM_LMAX];
  double redm[2][2 * HM_WARPS];
  double jac[HM_JAC_SMEM];
};

static __device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
static __device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
// FP32 operations of the running task: counted by thread 0 into s.bcast[7],
// collected by the executor after the task.
static __device__ __forceinline__ void count_f32(Smem& s, double f) {
  if (threadIdx.x == 0) s.bcast[7] += f;
}
static __device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide sum / max; result returned to every thread.
static __device__ __forceinline__ double block_sum(double v, Smem& s) {
  v = warp_sum(v);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) s.red[w] = v;
  __syncthreads();
  double r = 0.0;
#pragma unroll
  for (int i = 0; i < HM_WARPS; ++i) r += s.red[i];
  return r;
}
static __device__ __forceinline__ double block_max(double v, Smem& s) {
  v = warp_max(v);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) s.red[w] = v;
  __syncthreads();
  double r = 0.0;
#pragma unroll
  for (int i = 0; i < HM_WARPS; ++i) r = fmax(r, s.red[i]);
  return r;
}

// Set by set_status in the CTA whose error was the first recorded (the
// executor clears it before each task and reports that task's index).
static __shared__ int hm_status_won;

static __device__ __forceinline__ void set_status(int* status, int code) {
  if (atomicCAS(status, 0, code) == 0) hm_status_won = 1;
}

// ---------------------------------------------------------------------------
// One-sided Jacobi on J (p x c, ld p, p >= c) with accumulated rotations
// Vr (c x c, ld c): on return J's columns are mutually orthogonal and
// J_in Vr = J_out.
// ---------------------------------------------------------------------------
// s.ivals[2] receives the sweeps run, s.ivals[3] the rotations applied.
// A column whose squared norm is at most 1e-30 ||J||_F^2 (singular values
// below 1e-15 of the largest) is left alone: rotating it against the others
// changes no singular value above that level, and orthogonalising such
// rounding-level columns to relative accuracy is what made the sweeps many
// (the same cut-off as the one-sided Jacobi of LAPACK's xGESVJ for small
// columns).
template <class T>
static __device__ void cta_jacobi_t(T* J, int p, int c, T* Vr, Smem& s, T tol) {
  int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int idx = tid; idx < c * c; idx += HM_THREADS) Vr[idx] = (idx % c == idx / c) ? T(1) : T(0);
  if (tid == 0) {
    s.ivals[2] = 0;
    s.ivals[3] = 0;
  }
  double fro = 0.0;
  for (int idx = tid; idx < p * c; idx += HM_THREADS) fro += (double)J[idx] * (double)J[idx];
  const T negl = (T)(1e-30 * block_sum(fro, s));
  __syncthreads();
  if (c < 2) return;
  int N = c + (c & 1);
  for (int sweep = 0; sweep < 60; ++sweep) {
    if (tid == 0) {
      s.ivals[0] = 0;
      s.ivals[2] += 1;
    }
    __syncthreads();
    for (int r = 0; r < N - 1; ++r) {
      for (int k = warp; k < N / 2; k += HM_WARPS) {
        int a, b;
        if (k == 0) {
          a = r;
          b = N - 1;
        } else {
          a = (r + k) % (N - 1);
          b = (r - k + (N - 1)) % (N - 1);
        }
        if (a > b) {
          int t = a;
          a = b;
          b = t;
        }
        if (b >= c) continue;
        T* ja = J + (int64_t)a * p;
        T* jb = J + (int64_t)b * p;
        T al = T(0), be = T(0), ga = T(0);
        for (int i = lane; i < p; i += 32) {
          T x = ja[i], y = jb[i];
          al += x * x;
          be += y * y;
          ga += x * y;
        }
        al = warp_sum(al);
        be = warp_sum(be);
        ga = warp_sum(ga);
        if (al <= negl || be <= negl) continue;
        if (fabs(ga) <= tol * sqrt(al) * sqrt(be)) continue;
        T zeta = (be - al) / (T(2) * ga);
        T t = (zeta >= T(0) ? T(1) : T(-1)) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
        T cs = T(1) / sqrt(T(1) + t * t);
        T sn = cs * t;
        for (int i = lane; i < p; i += 32) {
          T x = ja[i], y = jb[i];
          ja[i] = cs * x - sn * y;
          jb[i] = sn * x + cs * y;
        }
        T* va = Vr + (int64_t)a * c;
        T* vb = Vr + (int64_t)b * c;
        for (int i = lane; i < c; i += 32) {
          T x = va[i], y = vb[i];
          va[i] = cs * x - sn * y;
          vb[i] = sn * x + cs * y;
        }
        if (lane == 0) {
          s.ivals[0] = 1;
          atomicAdd(&s.ivals[3], 1);
        }
      }
      __syncthreads();
    }
    int rotated = s.ivals[0];
    __syncthreads();
    if (!rotated) break;
  }
}

static __device__ void cta_jacobi(double* J, int p, int c, double* Vr, Smem& s, double tol = 1e-15) {
  cta_jacobi_t<double>(J, p, c, Vr, s, tol);
}

static __device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
static __device__ __forceinline__ float warp_max_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// One-sided Jacobi in FP32 (J p x c, ld p; rotations into Vr c x c): each
// pair of columns is handled by 16 lanes, so the 16 half-warps of the CTA
// take all pairs of a round-robin round (c <= 32) in one pass.  A pair is
// left alone once |a.b| <= tol |a| |b|.  The rank accounting of the callers
// is exact for any orthonormal Vr, so tol only decides how close the column
// norms come to the singular values (1e-4: closer than any rank decision
// needs); sweeps are capped at max_sweeps.
static __device__ void cta_jacobi_f(float* J, int p, int c, float* Vr, Smem& s, float tol, int max_sweeps) {
  int tid = threadIdx.x, hl = tid & 15, hw = tid >> 4;
  const int NHW = HM_THREADS / 16;
  unsigned mask = (tid & 16) ? 0xFFFF0000u : 0x0000FFFFu;
  for (int idx = tid; idx < c * c; idx += HM_THREADS) Vr[idx] = (idx % c == idx / c) ? 1.f : 0.f;
  if (tid == 0) {
    s.ivals[2] = 0;
    s.ivals[3] = 0;
  }
  __syncthreads();
  if (c < 2) return;
  int N = c + (c & 1);
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (tid == 0) {
      s.ivals[0] = 0;
      s.ivals[2] += 1;
    }
    __syncthreads();
    for (int r = 0; r < N - 1; ++r) {
      for (int k = hw; k < N / 2; k += NHW) {
        int a, b;
        if (k == 0) {
          a = r;
          b = N - 1;
        } else {
          a = (r + k) % (N - 1);
          b = (r - k + (N - 1)) % (N - 1);
        }
        if (a > b) {
          int t = a;
          a = b;
          b = t;
        }
        if (b >= c) continue;
        float* ja = J + (int64_t)a * p;
        float* jb = J + (int64_t)b * p;
        float al = 0.f, be = 0.f, ga = 0.f;
        for (int i = hl; i < p; i += 16) {
          float x = ja[i], y = jb[i];
          al += x * x;
          be += y * y;
          ga += x * y;
        }
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) {
          al += __shfl_xor_sync(mask, al, o);
          be += __shfl_xor_sync(mask, be, o);
          ga += __shfl_xor_sync(mask, ga, o);
        }
        if (al == 0.f || be == 0.f) continue;
        if (fabsf(ga) <= tol * sqrtf(al) * sqrtf(be)) continue;
        float zeta = (be - al) / (2.f * ga);
        float t = (zeta >= 0.f ? 1.f : -1.f) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
        float cs = 1.f / sqrtf(1.f + t * t);
        float sn = cs * t;
        for (int i = hl; i < p; i += 16) {
          float x = ja[i], y = jb[i];
          ja[i] = cs * x - sn * y;
          jb[i] = sn * x + cs * y;
        }
        float* va = Vr + (int64_t)a * c;
        float* vb = Vr + (int64_t)b * c;
        for (int i = hl; i < c; i += 16) {
          float x = va[i], y = vb[i];
          va[i] = cs * x - sn * y;
          vb[i] = sn * x + cs * y;
        }
        if (hl == 0) {
          s.ivals[0] = 1;
          atomicAdd(&s.ivals[3], 1);
        }
      }
      __syncthreads();
    }
    int rotated = s.ivals[0];
    __syncthreads();
    if (!rotated) break;
  }
}

// ---------------------------------------------------------------------------
// Row-parallel Householder factorisations (FP32 and FP64).  Row i of a panel
// belongs to thread i mod HM_THREADS for the whole factorisation, so the
// panel itself needs no barrier between steps; what crosses rows (the
// column's largest entry and sum of squares, the products v^T x_c with the
// trailing columns) is summed per warp and then over the warps in shared
// memory.  Each thread works on up to HM_QCH columns at once, so a tall
// panel in global memory has many independent loads in flight instead of one
// dependent chain per warp.  Conventions: column j becomes the reflector v_j
// (v_j[j] explicit, the rest below it), tau[j] = 2 / (v_j . v_j), rdiag[j]
// the diagonal of R, R above the diagonal in place.
// ---------------------------------------------------------------------------
#define HM_QCH 8

// first row >= j that belongs to this thread
static __device__ __forceinline__ int own_row(int j) {
  int t = threadIdx.x;
  return t >= j ? t : t + ((j - t + HM_THREADS - 1) / HM_THREADS) * HM_THREADS;
}

template <class T>
struct QrLimits;
template <>
struct QrLimits<float> {
  static __device__ __forceinline__ float zero() { return 1e-30f; }  // nothing left in a column below this
  static __device__ __forceinline__ float lo() { return 1e-10f; }    // squares safe between lo and hi
  static __device__ __forceinline__ float hi() { return 1e15f; }
};
template <>
struct QrLimits<double> {
  static __device__ __forceinline__ double zero() { return 1e-290; }
  static __device__ __forceinline__ double lo() { return 1e-140; }
  static __device__ __forceinline__ double hi() { return 1e140; }
};

static __device__ __forceinline__ float wsum(float v) { return warp_sum_f(v); }
static __device__ __forceinline__ double wsum(double v) { return warp_sum(v); }
static __device__ __forceinline__ float wmax(float v) { return warp_max_f(v); }
static __device__ __forceinline__ double wmax(double v) { return warp_max(v); }

// reduction buffers of the row-parallel factorisations, typed
template <class T>
static __device__ __forceinline__ T* qr_red(Smem& s, int b) {
  return reinterpret_cast<T*>(s.redd[b]);
}
template <class T>
static __device__ __forceinline__ T* qr_redm(Smem& s, int b) {
  return reinterpret_cast<T*>(s.redm[b]);
}

template <class T>
struct Refl {
  T tau, v0n, alpha;
};

// Reflector of column j from x0 = X(j, j) and the largest entry mx and the
// sum of squares sq of the rows below j (both already summed over the CTA).
// A column with nothing left gets tau = 0.  Entries so small (or so large)
// that their squares leave the floating-point range are first scaled in
// place by the column's largest entry (each thread its rows), with the sum
// taken again.
template <class T>
static __device__ Refl<T> reflector_t(T* xj, int j, int rows, T x0, T mx, T sq, Smem& s) {
  Refl<T> r;
  T ma = fmax(mx, fabs(x0));
  if (ma < QrLimits<T>::zero()) {
    r.tau = T(0);
    r.v0n = T(0);
    r.alpha = T(0);
    return r;
  }
  T scale = T(1);
  if (ma < QrLimits<T>::lo() || ma > QrLimits<T>::hi()) {
    T inv = T(1) / ma;
    T t = T(0);
    for (int i = own_row(j + 1); i < rows; i += HM_THREADS) {
      T v = xj[i] * inv;
      xj[i] = v;
      t += v * v;
    }
    sq = (T)block_sum((double)t, s);
    x0 *= inv;
    scale = ma;
  }
  T xn = sqrt(sq + x0 * x0);
  T alpha = x0 >= T(0) ? -xn : xn;
  r.v0n = x0 - alpha;
  r.tau = T(2) / (sq + r.v0n * r.v0n);
  r.alpha = alpha * scale;
  return r;
}

// Block totals of (max, sum of squares) partials through redm[b]; every
// thread gets the totals.  One barrier.
template <class T>
static __device__ __forceinline__ void block_max_sq(T& pm, T& ps, int b, Smem& s) {
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T* rm = qr_redm<T>(s, b);
  pm = wmax(pm);
  ps = wsum(ps);
  if (lane == 0) {
    rm[warp] = pm;
    rm[HM_WARPS + warp] = ps;
  }
  __syncthreads();
  pm = T(0);
  ps = T(0);
#pragma unroll
  for (int w = 0; w < HM_WARPS; ++w) {
    pm = fmax(pm, rm[w]);
    ps += rm[HM_WARPS + w];
  }
}

// Per-warp partial products d_c = v_j . x_{c0 + cc} (rows >= j) of a chunk
// of up to HM_QCH trailing columns into red (warp-major, HM_LMAX per warp).
template <class T>
static __device__ __forceinline__ void chunk_dots(const T* xj, T v0n, int j, int rows, const T* Xc, int ld, int nc,
                                                  T* red, int slot) {
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T d[HM_QCH];
#pragma unroll
  for (int cc = 0; cc < HM_QCH; ++cc) d[cc] = T(0);
  for (int i = own_row(j); i < rows; i += HM_THREADS) {
    T v = i == j ? v0n : xj[i];
    const T* xc = Xc + i;
#pragma unroll
    for (int cc = 0; cc < HM_QCH; ++cc)
      if (cc < nc) d[cc] += v * xc[(int64_t)cc * ld];
  }
#pragma unroll
  for (int cc = 0; cc < HM_QCH; ++cc) {
    T t = wsum(d[cc]);
    if (lane == 0 && cc < nc) red[warp * HM_LMAX + slot + cc] = t;
  }
}

// Totals of a chunk's partial products, times tau.
template <class T>
static __device__ __forceinline__ void chunk_totals(const T* red, int slot, int nc, T tau, T* d) {
#pragma unroll
  for (int cc = 0; cc < HM_QCH; ++cc) {
    T t = T(0);
    if (cc < nc)
#pragma unroll
      for (int w = 0; w < HM_WARPS; ++w) t += red[w * HM_LMAX + slot + cc];
    d[cc] = t * tau;
  }
}

// Householder QR of a panel X (rows x cols, ld), row-parallel, two barriers
// per column.  tau and rdiag may live in global or shared memory.
template <class T>
static __device__ void cta_qr_rows(T* X, int ld, int rows, int cols, double* tau, double* rdiag, Smem& s) {
  int tid = threadIdx.x;
  int q = rows < cols ? rows : cols;
  __syncthreads();
  if (q <= 0) return;
  T* red = qr_red<T>(s, 0);
  T pm = T(0), ps = T(0);
  for (int i = own_row(1); i < rows; i += HM_THREADS) {
    T x = X[i];
    pm = fmax(pm, fabs(x));
    ps += x * x;
  }
  T last_v0n = T(0);
  bool last_pending = false;
  for (int j = 0; j < q; ++j) {
    T* xj = X + (int64_t)j * ld;
    block_max_sq(pm, ps, j & 1, s);
    Refl<T> r = reflector_t(xj, j, rows, xj[j], pm, ps, s);
    if (tid == 0) {
      tau[j] = (double)r.tau;
      rdiag[j] = (double)r.alpha;
    }
    pm = T(0);
    ps = T(0);
    int nt = cols - j - 1;
    if (r.tau != T(0) && nt > 0) {
      for (int c0 = 0; c0 < nt; c0 += HM_QCH)
        chunk_dots(xj, r.v0n, j, rows, X + (int64_t)(j + 1 + c0) * ld, ld, min(HM_QCH, nt - c0), red, c0);
      __syncthreads();
      for (int c0 = 0; c0 < nt; c0 += HM_QCH) {
        int nc = min(HM_QCH, nt - c0);
        T d[HM_QCH];
        chunk_totals(red, c0, nc, r.tau, d);
        T* Xc = X + (int64_t)(j + 1 + c0) * ld;
        for (int i = own_row(j); i < rows; i += HM_THREADS) {
          T v = i == j ? r.v0n : xj[i];
#pragma unroll
          for (int cc = 0; cc < HM_QCH; ++cc) {
            if (cc < nc) {
              T x = Xc[(int64_t)cc * ld + i] - d[cc] * v;
              Xc[(int64_t)cc * ld + i] = x;
              if (c0 + cc == 0 && i > j + 1) {
                pm = fmax(pm, fabs(x));
                ps += x * x;
              }
            }
          }
        }
      }
      if (own_row(j) == j) xj[j] = r.v0n;  // every thread has read X(j, j)
    } else {
      // a zero column (nothing to apply) or the last column: the next
      // column's partials from its rows as they are; the last column's
      // explicit first entry is written after the final barrier
      if (j + 1 < q) {
        const T* xn = X + (int64_t)(j + 1) * ld;
        for (int i = own_row(j + 2); i < rows; i += HM_THREADS) {
          T x = xn[i];
          pm = fmax(pm, fabs(x));
          ps += x * x;
        }
      }
      last_pending = r.tau != T(0);
      last_v0n = r.v0n;
    }
  }
  __syncthreads();
  if (last_pending && own_row(q - 1) == q - 1) X[(int64_t)(q - 1) * ld + q - 1] = last_v0n;
  __syncthreads();
}

// Y (rows x k, ldy) <- P_0 P_1 ... P_{q-1} Y with the reflectors of a
// row-parallel QR in V (tau as it left it), row-parallel: the reflectors are
// applied in reverse order, one barrier each.
template <class T>
static __device__ void cta_apply_q_rows(const T* V, int ldv, int rows, int q, const double* tau, T* Y, int ldy, int k,
                                        Smem& s) {
  __syncthreads();
  for (int j = q - 1; j >= 0; --j) {
    T tj = (T)tau[j];
    if (tj == T(0) || k <= 0) continue;
    const T* vj = V + (int64_t)j * ldv;
    T v0 = vj[j];
    T* red = qr_red<T>(s, j & 1);
    for (int c0 = 0; c0 < k; c0 += HM_QCH)
      chunk_dots(vj, v0, j, rows, Y + (int64_t)c0 * ldy, ldy, min(HM_QCH, k - c0), red, c0);
    __syncthreads();
    for (int c0 = 0; c0 < k; c0 += HM_QCH) {
      int nc = min(HM_QCH, k - c0);
      T d[HM_QCH];
      chunk_totals(red, c0, nc, tj, d);
      T* Yc = Y + (int64_t)c0 * ldy;
      for (int i = own_row(j); i < rows; i += HM_THREADS) {
        T v = vj[i];
#pragma unroll
        for (int cc = 0; cc < HM_QCH; ++cc)
          if (cc < nc) Yc[(int64_t)cc * ldy + i] -= d[cc] * v;
      }
    }
  }
  __syncthreads();
}

static __device__ void cta_qr_f(float* X, int ld, int rows, int cols, double* tau, double* rdiag, Smem& s) {
  cta_qr_rows<float>(X, ld, rows, cols, tau, rdiag, s);
}
static __device__ void cta_apply_qf(const float* V, int ldv, int rows, int q, const double* tau, float* Y, int ldy,
                                    int k, Smem& s) {
  cta_apply_q_rows<float>(V, ldv, rows, q, tau, Y, ldy, k, s);
}

// Q = P_0 ... P_{q-1} [I; 0] (rows x q, ld ldq) from the reflectors of a
// row-parallel FP32 QR.
static __device__ void form_q_f(const float* V, int ldv, int rows, int q, const double* tau, float* Q, int ldq,
                                Smem& s) {
  __syncthreads();
  for (int c = 0; c < q; ++c)
    for (int i = threadIdx.x; i < rows; i += HM_THREADS) Q[(int64_t)c * ldq + i] = (i == c) ? 1.f : 0.f;
  cta_apply_qf(V, ldv, rows, q, tau, Q, ldq, q, s);
}

// Column-pivoted Householder QR of a float panel, X P = Q R, row-parallel
// (conventions of cta_qr_f; perm[j] = the original column now at j).  The
// pivot is the trailing column of largest remaining norm; those norms are
// summed afresh at every step from the updated rows (no downdating), so
// every thread takes the same pivot from the same shared sums.  Three
// barriers per column.
static __device__ void cta_qrcp_f(float* X, int ld, int rows, int cols, double* tau, double* rdiag, int* perm,
                                  Smem& s) {
  int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int q = rows < cols ? rows : cols;
  float* dred = qr_red<float>(s, 0);  // partial products with the reflector
  float* nred = qr_red<float>(s, 1);  // partial squared norms of the trailing columns
  __syncthreads();
  for (int c = tid; c < cols; c += HM_THREADS) perm[c] = c;
  // squared norms of the whole columns
  for (int c0 = 0; c0 < cols; c0 += HM_QCH) {
    int nc = min(HM_QCH, cols - c0);
    float d[HM_QCH];
#pragma unroll
    for (int cc = 0; cc < HM_QCH; ++cc) d[cc] = 0.f;
    for (int i = tid; i < rows; i += HM_THREADS)
#pragma unroll
      for (int cc = 0; cc < HM_QCH; ++cc)
        if (cc < nc) {
          float x = X[(int64_t)(c0 + cc) * ld + i];
          d[cc] += x * x;
        }
#pragma unroll
    for (int cc = 0; cc < HM_QCH; ++cc) {
      float t = wsum(d[cc]);
      if (lane == 0 && cc < nc) nred[warp * HM_LMAX + c0 + cc] = t;
    }
  }
  __syncthreads();
  for (int j = 0; j < q; ++j) {
    // pivot: the same scan of the same sums on every thread
    int pv = j;
    float best = -1.f;
    for (int c = j; c < cols; ++c) {
      float t = 0.f;
#pragma unroll
      for (int w = 0; w < HM_WARPS; ++w) t += nred[w * HM_LMAX + c];
      if (t > best) {
        best = t;
        pv = c;
      }
    }
    float* xj = X + (int64_t)j * ld;
    float pm = 0.f, ps = 0.f;
    if (pv != j) {
      float* xp = X + (int64_t)pv * ld;
      for (int i = tid; i < rows; i += HM_THREADS) {
        float a = xj[i], b = xp[i];
        xj[i] = b;
        xp[i] = a;
        if (i > j) {
          pm = fmaxf(pm, fabsf(b));
          ps += b * b;
        }
      }
    } else {
      for (int i = own_row(j + 1); i < rows; i += HM_THREADS) {
        float x = xj[i];
        pm = fmaxf(pm, fabsf(x));
        ps += x * x;
      }
    }
    block_max_sq(pm, ps, j & 1, s);  // also: every thread is past its pivot scan
    if (tid == 0 && pv != j) {
      int u = perm[j];
      perm[j] = perm[pv];
      perm[pv] = u;
    }
    Refl<float> r = reflector_t(xj, j, rows, xj[j], pm, ps, s);
    if (tid == 0) {
      tau[j] = r.tau;
      rdiag[j] = r.alpha;
    }
    int nt = cols - j - 1;
    if (r.tau != 0.f && nt > 0) {
      for (int c0 = 0; c0 < nt; c0 += HM_QCH)
        chunk_dots(xj, r.v0n, j, rows, X + (int64_t)(j + 1 + c0) * ld, ld, min(HM_QCH, nt - c0), dred, c0);
      __syncthreads();
    }
    // update the trailing columns and sum their squared norms below row j
    for (int c0 = 0; c0 < nt; c0 += HM_QCH) {
      int nc = min(HM_QCH, nt - c0);
      float d[HM_QCH], sq[HM_QCH];
      if (r.tau != 0.f) chunk_totals(dred, c0, nc, r.tau, d);
#pragma unroll
      for (int cc = 0; cc < HM_QCH; ++cc) sq[cc] = 0.f;
      float* Xc = X + (int64_t)(j + 1 + c0) * ld;
      for (int i = own_row(j); i < rows; i += HM_THREADS) {
        float v = i == j ? r.v0n : xj[i];
#pragma unroll
        for (int cc = 0; cc < HM_QCH; ++cc) {
          if (cc < nc) {
            float x = Xc[(int64_t)cc * ld + i];
            if (r.tau != 0.f) {
              x -= d[cc] * v;
              Xc[(int64_t)cc * ld + i] = x;
            }
            if (i > j) sq[cc] += x * x;
          }
        }
      }
#pragma unroll
      for (int cc = 0; cc < HM_QCH; ++cc) {
        float t = wsum(sq[cc]);
        if (lane == 0 && cc < nc) nred[warp * HM_LMAX + j + 1 + c0 + cc] = t;
      }
    }
    __syncthreads();  // the next pivot scan reads the new sums
    if (r.tau != 0.f && own_row(j) == j) xj[j] = r.v0n;
  }
  __syncthreads();
}


static __device__ void cta_order_sigma(int c, Smem& s);
// Column norms of J into sigma, and the order of decreasing sigma into order.
static __device__ void cta_sort_sigma(const double* J, int p, int c, Smem& s) {
  int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int j = warp; j < c; j += HM_WARPS) {
    const double* jj = J + (int64_t)j * p;
    double x = 0.0;
    for (int i = lane; i < p; i += 32) x += jj[i] * jj[i];
    x = warp_sum(x);
    if (lane == 0) s.sigma[j] = sqrt(x);
  }
  __syncthreads();
  cta_order_sigma(c, s);
}

// The order of decreasing s.sigma[0..c) into s.order (ties by index).
static __device__ void cta_order_sigma(int c, Smem& s) {
  int tid = threadIdx.x;
  for (int j = tid; j < c; j += HM_THREADS) {
    double sj = s.sigma[j];
    int rk = 0;
    for (int i = 0; i < c; ++i) {
      double si = s.sigma[i];
      rk += (si > sj) || (si == sj && i < j);
    }
    s.order[rk] = j;
  }
  __syncthreads();
}

// "Choose new rank k": smallest k with sum_{i>k} s_i^2 <= eps^2 sum_i s_i^2
// (rule 0, relative Frobenius), or the number of s_i > eps s_1 (rule 1,
// relative spectral).
static __device__ int cta_choose_rank(int c, double eps, Smem& s, int rule = 0) {
  if (threadIdx.x == 0 && rule == 1) {
    double s1 = c > 0 ? s.sigma[s.order[0]] : 0.0;
    int k = 0;
    while (k < c && s.sigma[s.order[k]] > eps * s1) ++k;
    s.ivals[1] = k;
  } else if (threadIdx.x == 0) {
    double total = 0.0;
    for (int i = 0; i < c; ++i) {
      double x = s.sigma[s.order[i]];
      total += x * x;
    }
    double bound = eps * eps * total;
    double tail = 0.0;
    int k = c;
    while (k > 0) {
      double x = s.sigma[s.order[k - 1]];
      if (tail + x * x <= bound) {
        tail += x * x;
        --k;
      } else {
        break;
      }
    }
    s.ivals[1] = k;
  }
  __syncthreads();
  int k = s.ivals[1];
  __syncthreads();
  return k;
}

// ---------------------------------------------------------------------------
// Truncation core (Section 3 "Truncation", Fig. rkadd, Fig. rowmerge).
//
// R = sum_j SA_j SB_j^T with nb (1 or 2) blocks; block j has SA_j (m x k_j,
// ld m) and SB_j (n_j x k_j, ld n_j), the SB_j stacked (rows n_0 then n_1) in
// the result.  nb = 1 is rkadd on the stacked factors, nb = 2 is rowmerge.
// SB_j are overwritten (QR reflectors).  W is scratch of m x (sum q_j).
// Result: U (m x k, ld ldu) = left singular vectors, V (sum n_j x k, ld ldv)
// = right singular vectors times singular values; k returned (<= cap).
// ---------------------------------------------------------------------------
struct TruncIn {
  int nb;
  int m;
  int n[2];
  int k[2];
  const double* SA[2];
  double* SB[2];
  double* W;        // m x (q0 + q1)
  double* Jg;       // global fallback for the Jacobi core (p*c + c*c doubles)
};

// Householder QR flops of a rows x cols matrix (Golub & Van Loan count).
static __device__ __forceinline__ double qr_flops(double rows, double cols) {
  return rows >= cols ? 2.0 * cols * cols * (rows - cols / 3.0) : 2.0 * rows * rows * (cols - rows / 3.0);
}

static __device__ int trunc_core(const TruncIn& in, double eps, int cap, double* U, int ldu, double* V, int ldv,
                          int* status, Smem& s, double* flops = nullptr, int rule = 0) {
  int tid = threadIdx.x;
  int m = in.m;
  int q[2] = {0, 0};
  int qoff[2] = {0, 0};
  for (int j = 0; j < in.nb; ++j) q[j] = in.n[j] < in.k[j] ? in.n[j] : in.k[j];
  qoff[1] = q[0];
  int qs = q[0] + (in.nb > 1 ? q[1] : 0);
  // tauB / rdiagB hold both blocks' reflectors at offsets qoff.
  for (int j = 0; j < in.nb; ++j)
    cta_qr_rows<double>(in.SB[j], in.n[j], in.n[j], in.k[j], s.tauB + qoff[j], s.rdiagB + qoff[j], s);
  if (m == 0 || qs == 0) return 0;
  // Ahat = [SA_0 R_0^T, SA_1 R_1^T]  (m x qs)
  for (int j = 0; j < in.nb; ++j) {
    const double* SA = in.SA[j];
    const double* SB = in.SB[j];
    int nj = in.n[j], kj = in.k[j];
    for (int idx = tid; idx < m * q[j]; idx += HM_THREADS) {
      int r = idx % m, i = idx / m;
      double acc = SA[(int64_t)i * m + r] * s.rdiagB[qoff[j] + i];
      for (int c = i + 1; c < kj; ++c) acc += SA[(int64_t)c * m + r] * SB[(int64_t)c * nj + i];
      in.W[(int64_t)(qoff[j] + i) * m + r] = acc;
    }
  }
  __syncthreads();
  // QR of Ahat
  cta_qr_rows<double>(in.W, m, m, qs, s.tauA, s.rdiagA, s);
  int qa = m < qs ? m : qs;
  // Jacobi core: case A (qa == qs): J = R_A (qs x qs); case B: J = R_A^T (qs x qa)
  bool caseA = (qa == qs);
  int p = caseA ? qs : qs;
  int c = caseA ? qs : qa;
  double* J;
  double* Vr;
  if ((int64_t)p * c + (int64_t)c * c <= HM_JAC_SMEM) {
    J = s.jac;
  } else {
    J = in.Jg;
  }
  Vr = J + (int64_t)p * c;
  for (int idx = tid; idx < p * c; idx += HM_THREADS) {
    int i = idx % p, j = idx / p;
    // R_A(row, col) with row < qa, col < qs
    int row = caseA ? i : j, col = caseA ? j : i;
    double v;
    if (row > col) v = 0.0;
    else if (row == col) v = s.rdiagA[row];
    else v = in.W[(int64_t)col * m + row];
    J[idx] = v;
  }
  __syncthreads();
  cta_jacobi(J, p, c, Vr, s);
  cta_sort_sigma(J, p, c, s);
  int k = cta_choose_rank(c, eps, s, rule);
  if (flops && tid == 0) {
    double f = 0.0;
    for (int j = 0; j < in.nb; ++j) {
      f += qr_flops(in.n[j], in.k[j]);                       // QR of the stacked B factors
      f += (double)m * q[j] * (2.0 * in.k[j] - q[j]);        // Ahat = A R^T (triangular)
      f += 4.0 * in.n[j] * q[j] * (k < cap ? k : cap);       // V = Q_B (Vhat Sigma)
    }
    f += qr_flops(m, qs);                                    // QR of Ahat
    f += (double)s.ivals[2] * 0.5 * c * (c - 1) * 6.0 * p;   // Jacobi: column products per sweep
    f += (double)s.ivals[3] * 6.0 * (p + c);                 // Jacobi: rotations
    f += 4.0 * m * qa * (k < cap ? k : cap);                 // U = Q_A U_c
    *flops += f;
  }
  if (k > cap) {
    if (tid == 0) set_status(status, DS_RANK);
    k = cap;
  }
  // Left factor: U = Q_A [left(:, order[0:k]); 0]
  for (int idx = tid; idx < m * k; idx += HM_THREADS) {
    int r = idx % m, jj = idx / m;
    int col = s.order[jj];
    double v = 0.0;
    if (r < qa) {
      if (caseA) {
        double sg = s.sigma[col];
        v = sg > 0.0 ? J[(int64_t)col * p + r] / sg : 0.0;
      } else {
        v = Vr[(int64_t)col * c + r];
      }
    }
    U[(int64_t)jj * ldu + r] = v;
  }
  // Right factor per block j: V_j = Q_j [right(qoff_j : qoff_j + q_j, order) * sigma; 0]
  int voff = 0;
  for (int j = 0; j < in.nb; ++j) {
    int nj = in.n[j];
    for (int idx = tid; idx < nj * k; idx += HM_THREADS) {
      int r = idx % nj, jj = idx / nj;
      int col = s.order[jj];
      double v = 0.0;
      if (r < q[j]) {
        int rr = qoff[j] + r;
        if (caseA) v = Vr[(int64_t)col * c + rr] * s.sigma[col];
        else v = J[(int64_t)col * p + rr];
      }
      V[(int64_t)jj * ldv + voff + r] = v;
    }
    voff += nj;
  }
  __syncthreads();
  cta_apply_q_rows<double>(in.W, m, m, qa, s.tauA, U, ldu, k, s);
  voff = 0;
  for (int j = 0; j < in.nb; ++j) {
    cta_apply_q_rows<double>(in.SB[j], in.n[j], in.n[j], q[j], s.tauB + qoff[j], V + voff, ldv, k, s);
    voff += in.n[j];
  }
  return k;
}

// ---------------------------------------------------------------------------
// Randomised truncation: the range finder of Halko, Martinsson and Tropp
// (SIAM Review 2011, Alg. 4.1) with an exact a-posteriori check of the
// truncation rule.  M (m x n) is given explicitly (Md, ld m) or as SA SB^T
// (m x l, n x l).  For a sketch width r:
//   Y = M Omega            (Rademacher Omega, FP32 -- only picks a subspace)
//   Q = orth(Y)            (FP64 Householder, explicit m x r)
//   J = M^T Q = (Q^T M)^T  (FP64)
//   one-sided Jacobi on J  -> singular triplets of Q^T M (FP64), or for
//                            eps >= HM_F32_MIN_EPS the FP32 core of
//                            core_f32 (pivoted QR, a few sweeps on R^T)
//   res^2 = ||M||_F^2 - ||Q^T M||_F^2  (FP64, exact for orthonormal Q)
// The rank k is the smallest with res^2 + sum_{i>k} sigma_i^2 <= eps^2 ||M||_F^2,
// so the result meets the same Frobenius rule as the exact truncation (its
// rank can exceed the optimal one by what the subspace missed).  If even
// k = r fails, r doubles up to rmax; then the caller falls back to the exact
// QR + SVD path.  C = Q Vr(:, order), D = J(:, order) as in Fig. rkadd.
// ---------------------------------------------------------------------------
#define HM_RMAX 32
#ifndef HM_CORE_SWEEPS
#define HM_CORE_SWEEPS 2  // Jacobi sweeps on the pivoted R^T of the FP32 core
#endif
#define HM_F32_MIN_EPS 1e-5  // FP32 rounding (~1e-7) stays well below eps from here on

struct RandIn {
  int m, n, l;
  const double* Md;   // explicit M (ld m) or nullptr
  const double* SA;   // m x l (ld m)
  const double* SB;   // n x l (ld n)
  double* ws;         // rand_ws_doubles(m, n, l) doubles
  uint64_t seed;
  int r0;             // first sketch width
};

static __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Orthonormal C for the kept part of a core_f32 result: the kept columns of
// W (in decreasing order of norm) are factored Wk = Wh T (FP32 Householder,
// Wh explicit in r x k), and Z = Vrot(:, kept) T^T (r x k, written over W),
// so that (P W_k)(Q_J Vrot_k)^T = (P Wh)(Q_J Z)^T with P Wh orthonormal.
// Wk, Wh: r x k floats each, apart from cw.
static __device__ void core_f32_orth(float* cw, int r, int k, float* Wk, float* Wh, Smem& s) {
  int tid = threadIdx.x;
  const float* W = cw;
  const float* Vrot = cw + r * r;
  for (int idx = tid; idx < r * k; idx += HM_THREADS) {
    int i = idx % r, jj = idx / r;
    Wk[idx] = W[i + (int64_t)s.order[jj] * r];
  }
  cta_qr_f(Wk, r, r, k, s.tauA, s.rdiagA, s);
  form_q_f(Wk, r, r, k, s.tauA, Wh, r, s);
  float* Z = cw;
  for (int idx = tid; idx < r * k; idx += HM_THREADS) {
    int j = idx % r, jj = idx / r;
    float z = 0.f;
    for (int q = jj; q < k; ++q) {
      float t = q == jj ? (float)s.rdiagA[jj] : Wk[(int64_t)q * r + jj];
      z += Vrot[j + (int64_t)s.order[q] * r] * t;
    }
    Z[idx] = z;
  }
  __syncthreads();
}

// Small core of the FP32 randomised truncations.  J (p x r floats, ld p, p >= r) is
// factored in place, J P = Q_J R (cta_qrcp_f; reflectors and tau in s.tauB
// for forming Q_J); one-sided Jacobi on R^T, at most max_sweeps sweeps (the
// pivoted R^T has graded columns, so few sweeps come close to its SVD),
// gives R^T Vrot = W.  Out: W and Vrot (r x r, in cw: W, Vrot, then r floats
// of norms and r ints of perm), s.sigma = column norms of W, s.order = their
// decreasing order.  With J = Q_J R P^T = Q_J Vrot W^T P^T, dropping columns
// of W drops exactly their squared norms (Vrot and Q_J orthonormal).
static __device__ void core_f32(float* J, int p, int r, float* cw, Smem& s, int max_sweeps) {
  int tid = threadIdx.x;
  float* W = cw;
  float* Vrot = W + r * r;
  float* nrm = Vrot + r * r;
  int* perm = (int*)(nrm + r);
  cta_qrcp_f(J, p, p, r, s.tauB, s.rdiagB, perm, s);
  // X = R^T: X[i][c] = R[c][i], nonzero for c <= i
  for (int idx = tid; idx < r * r; idx += HM_THREADS) {
    int i = idx % r, c = idx / r;
    W[idx] = c > i ? 0.f : (c == i ? (float)s.rdiagB[i] : J[(int64_t)i * p + c]);
  }
  __syncthreads();
  cta_jacobi_f(W, r, r, Vrot, s, 1e-4f, max_sweeps);
  int lane = tid & 31, warp = tid >> 5;
  for (int j = warp; j < r; j += HM_WARPS) {
    float x = 0.f;
    for (int i = lane; i < r; i += 32) x += W[i + j * r] * W[i + j * r];
    x = warp_sum_f(x);
    if (lane == 0) s.sigma[j] = sqrt((double)x);
  }
  __syncthreads();
  cta_order_sigma(r, s);
}

static __device__ int trunc_rand(const RandIn& in, double eps, int cap, double* U, int ldu, double* V, int ldv,
                          int* status, Smem& s, double* flops, int* ok) {
  int tid = threadIdx.x;
  if (tid == 0) s.ivals[5] = s.ivals[6] = 0;  // attempts, columns sketched over all attempts
  int m = in.m, n = in.n, l = in.l;
  bool factored = (in.Md == nullptr);
  int rmax = HM_RMAX;
  if (rmax > m) rmax = m;
  if (rmax > n) rmax = n;
  if (factored && rmax > l) rmax = l;
  // Y (m x RMAX: sketch, then reflectors), Qx (m x RMAX), J (n x RMAX) and
  // Vr (RMAX x RMAX) live in shared memory when they fit (the sequential
  // steps of the QR and the Jacobi rounds then avoid L2 round trips), else in
  // the scratch.  Signs and Grams always use the scratch.
  bool in_smem = (int64_t)(2 * m + n) * rmax + (int64_t)rmax * rmax <= HM_JAC_SMEM;
  int R = in_smem ? rmax : HM_RMAX;
  double* Y = in_smem ? s.jac : in.ws;
  double* Qx = Y + (int64_t)m * R;
  double* J = Qx + (int64_t)m * R;
  double* Vr = J + (int64_t)n * R;
  double* gws = in.ws + (int64_t)(2 * m + n) * HM_RMAX + HM_RMAX * HM_RMAX;
  uint32_t* Om = (uint32_t*)gws;                          // n sign words
  double* G = gws + (n + 1) / 2 + 1;                       // 2 l x l Grams, or T (l x RMAX floats)
  int64_t gsz = 2 * (int64_t)l * l > (int64_t)l * HM_RMAX ? 2 * (int64_t)l * l : (int64_t)l * HM_RMAX;
  // FP32 core (eps >= HM_F32_MIN_EPS) after the Grams: J as floats (then its
  // reflectors), Q_J, and the core's W, Vrot, norms and permutation
  bool f32core = eps >= HM_F32_MIN_EPS;
  float* Jf = (float*)(G + gsz);                           // n x RMAX floats
  float* Qj = Jf + (int64_t)n * HM_RMAX;                   // n x RMAX floats
  float* cw = Qj + (int64_t)n * HM_RMAX;                   // 4 RMAX^2 + 2 RMAX
  double f = 0.0;
  // ||M||_F^2
  double total;
  if (!factored) {
    double acc = 0.0;
    for (int64_t idx = tid; idx < (int64_t)m * n; idx += HM_THREADS) {
      double x = in.Md[idx];
      acc += x * x;
    }
    total = block_sum(acc, s);
    f += 2.0 * m * n;
  } else {
    double* GA = G;
    double* GB = G + (int64_t)l * l;
    for (int idx = tid; idx < l * l; idx += HM_THREADS) {
      int i = idx % l, j = idx / l;
      double a = 0.0, b = 0.0;
      if (i <= j) {
        for (int r = 0; r < m; ++r) a += in.SA[(int64_t)i * m + r] * in.SA[(int64_t)j * m + r];
        for (int r = 0; r < n; ++r) b += in.SB[(int64_t)i * n + r] * in.SB[(int64_t)j * n + r];
      }
      GA[idx] = a;
      GB[idx] = b;
    }
    __syncthreads();
    double acc = 0.0;
    for (int idx = tid; idx < l * l; idx += HM_THREADS) {
      int i = idx % l, j = idx / l;
      if (i <= j) acc += (i == j ? 1.0 : 2.0) * GA[idx] * GB[idx];
    }
    total = block_sum(acc, s);
    f += (double)(m + n) * l * (l + 1);
  }
  double bound = eps * eps * total;
  if (total == 0.0) {
    *ok = 1;
    return 0;
  }
  int r = in.r0 < 2 ? 2 : in.r0;
  if (r > rmax) r = rmax;
  for (;;) {
    __syncthreads();
    if (tid == 0) {
      s.ivals[5] += 1;
      s.ivals[6] += r;
    }
    // Rademacher signs, one 32-bit word per row of Omega
    for (int i = tid; i < n; i += HM_THREADS) Om[i] = (uint32_t)mix64(in.seed ^ ((uint64_t)i * 0xD1B54A32D192ED03ull));
    __syncthreads();
    // sketch Y = M Omega in FP32
    if (!factored) {
      for (int idx = tid; idx < m * r; idx += HM_THREADS) {
        int i = idx % m, j = idx / m;
        float acc = 0.f;
        for (int c = 0; c < n; ++c) {
          float x = (float)in.Md[(int64_t)c * m + i];
          acc += ((Om[c] >> j) & 1u) ? x : -x;
        }
        Y[(int64_t)j * m + i] = (double)acc;
      }
    } else {
      float* T = (float*)G;  // l x r, reuses the Gram space (no longer needed)
      for (int idx = tid; idx < l * r; idx += HM_THREADS) {
        int i = idx % l, j = idx / l;
        float acc = 0.f;
        for (int c = 0; c < n; ++c) {
          float x = (float)in.SB[(int64_t)i * n + c];
          acc += ((Om[c] >> j) & 1u) ? x : -x;
        }
        T[idx] = acc;
      }
      __syncthreads();
      for (int idx = tid; idx < m * r; idx += HM_THREADS) {
        int i = idx % m, j = idx / m;
        float acc = 0.f;
        for (int c = 0; c < l; ++c) acc += (float)in.SA[(int64_t)c * m + i] * T[(int64_t)j * l + c];
        Y[(int64_t)j * m + i] = (double)acc;
      }
    }
    __syncthreads();
    // Q = orth(Y): Householder, then explicit Q = P_0 ... P_{r-1} [I; 0]
    int rr = r < m ? r : m;
    cta_qr_rows<double>(Y, m, m, r, s.tauA, s.rdiagA, s);
    for (int idx = tid; idx < m * rr; idx += HM_THREADS) Qx[idx] = (idx % m == idx / m) ? 1.0 : 0.0;
    __syncthreads();
    cta_apply_q_rows<double>(Y, m, m, rr, s.tauA, Qx, m, rr, s);
    // J = M^T Q (n x rr) in FP64
    if (!factored) {
      for (int idx = tid; idx < n * rr; idx += HM_THREADS) {
        int c = idx % n, j = idx / n;
        double acc = 0.0;
        for (int i = 0; i < m; ++i) acc += in.Md[(int64_t)c * m + i] * Qx[(int64_t)j * m + i];
        J[idx] = acc;
      }
      f += 2.0 * m * n * rr;
    } else {
      double* P = G;  // rr x l
      for (int idx = tid; idx < rr * l; idx += HM_THREADS) {
        int j = idx % rr, c = idx / rr;
        double acc = 0.0;
        for (int i = 0; i < m; ++i) acc += Qx[(int64_t)j * m + i] * in.SA[(int64_t)c * m + i];
        P[idx] = acc;
      }
      __syncthreads();
      for (int idx = tid; idx < n * rr; idx += HM_THREADS) {
        int c = idx % n, j = idx / n;
        double acc = 0.0;
        for (int i = 0; i < l; ++i) acc += in.SB[(int64_t)i * n + c] * P[(int64_t)i * rr + j];
        J[idx] = acc;
      }
      f += 2.0 * (m + n) * (double)l * rr;
    }
    __syncthreads();
    f += qr_flops(m, r) + 4.0 * m * rr * rr;
    double jn2 = 0.0;
    if (f32core) {
      // ||J||_F^2 in FP64 for the residual; the core (pivoted QR, a few
      // Jacobi sweeps on R^T) on an FP32 copy of J, then Q_J explicitly
      double a2 = 0.0;
      for (int idx = tid; idx < n * rr; idx += HM_THREADS) {
        double x = J[idx];
        a2 += x * x;
        Jf[idx] = (float)x;
      }
      jn2 = block_sum(a2, s);
      core_f32(Jf, n, rr, cw, s, HM_CORE_SWEEPS);
      form_q_f(Jf, n, n, rr, s.tauB, Qj, n, s);
      count_f32(s, 4.0 * n * rr * rr + 12.0 * rr * (double)s.ivals[3]);
      f += 2.0 * n * rr;
    } else {
      cta_jacobi(J, n, rr, Vr, s, 1e-10);
      cta_sort_sigma(J, n, rr, s);
      f += (double)s.ivals[2] * 0.5 * rr * (rr - 1) * 6.0 * n + (double)s.ivals[3] * 6.0 * (n + rr);
    }
    if (tid == 0) {
      double sum = 0.0;
      if (f32core) {
        sum = jn2;
      } else {
        for (int i = 0; i < rr; ++i) sum += s.sigma[i] * s.sigma[i];
      }
      double res2 = total - sum;
      if (res2 < 0.0) res2 = 0.0;
      int k = -1;
      if (res2 <= bound) {
        double tail = res2;
        k = rr;
        while (k > 0) {
          double x = s.sigma[s.order[k - 1]];
          if (tail + x * x <= bound) {
            tail += x * x;
            --k;
          } else {
            break;
          }
        }
      }
      s.ivals[4] = k;
    }
    __syncthreads();
    int k = s.ivals[4];
    __syncthreads();
    if (k < 0) {
      if (r >= rmax) {
        if (flops && tid == 0) *flops += f;
        *ok = 0;
        return 0;
      }
      r = 2 * r > rmax ? rmax : 2 * r;
      continue;
    }
    if (k > cap) {
      if (tid == 0) set_status(status, DS_RANK);
      k = cap;
    }
    float* Wk = cw + 2 * HM_RMAX * HM_RMAX + 2 * HM_RMAX;
    float* Wh = Wk + HM_RMAX * HM_RMAX;
    if (f32core && k > 0) core_f32_orth(cw, rr, k, Wk, Wh, s);
    for (int idx = tid; idx < m * k; idx += HM_THREADS) {
      int i = idx % m, jj = idx / m;
      int col = s.order[jj];
      double acc = 0.0;
      if (f32core) {
        const int* perm = (const int*)(cw + 2 * rr * rr + rr);
        for (int j = 0; j < rr; ++j) acc += Qx[(int64_t)perm[j] * m + i] * (double)Wh[(int64_t)jj * rr + j];
      } else
        for (int j = 0; j < rr; ++j) acc += Qx[(int64_t)j * m + i] * Vr[(int64_t)col * rr + j];
      U[(int64_t)jj * ldu + i] = acc;
    }
    for (int idx = tid; idx < n * k; idx += HM_THREADS) {
      int i = idx % n, jj = idx / n;
      int col = s.order[jj];
      if (f32core) {
        const float* zc = cw + (int64_t)jj * rr;
        float acc = 0.f;
        for (int j = 0; j < rr; ++j) acc += Qj[(int64_t)j * n + i] * zc[j];
        V[(int64_t)jj * ldv + i] = (double)acc;
      } else {
        V[(int64_t)jj * ldv + i] = J[(int64_t)col * n + i];
      }
    }
    f += 2.0 * m * rr * k;
    if (flops && tid == 0) *flops += f;
    *ok = 1;
    return k;
  }
}

// ---------------------------------------------------------------------------
// Mixed-precision randomised truncation of an explicit M (m x n, FP32 copy,
// ld m).  The sketch Y = M Omega, Q = orth(Y) and the projection J = M^T Q
// run in FP32; the residual ||M - Q J^T||_F^2 is formed entry by entry (FP32
// differences, FP64 sum), which stays accurate where the difference of the
// two squared norms would cancel.  The small core (core_f32): J P = Q_J R
// by pivoted QR, R^T Vrot = W by a few Jacobi sweeps, so that
// M ~ Q J^T = (Q P W)(Q_J Vrot)^T with Q_J Vrot orthonormal and
//   C = Q P W(:, order), D = Q_J Vrot(:, order)  (Fig. rkadd's C, D),
// the dropped columns of W costing exactly their squared norms.
// Rank rule as trunc_rand: res^2 + tail <= eps^2 ||M||_F^2.
// M arrives scaled by 1/scale (largest entry 1, clear of the FP32 range
// limits); the rule is scale invariant and D is multiplied back by scale.
// Float work space fw: 2 m R + 2 n R floats (R = min(32, m, n)); an attempt
// of width r uses its first 2 (m + n) r floats, or the first floats of s.jac
// when fw is global and they fit there; Om: n words; the core's W, Vrot
// (2 r^2 floats and 2 r words) sit at s.jac + HM_F32_SMEM / 2.
// ---------------------------------------------------------------------------
#define HM_G32_MB 64
#define HM_G32_NB 64
#define HM_G32_KB 32
#define HM_G32_LD 65  // padded row of a staged tile (odd: no bank conflicts either way)
#define HM_G32_SMEM (2 * HM_G32_KB * HM_G32_LD)  // floats of staging

// C (m x n, ldc) (+)= alpha op(A) op(B) as cta_gemm, with 64 x 64 output
// tiles, 32-deep FP32 operand tiles in sm (HM_G32_SMEM floats) and a 4 x 4
// register block per thread; C may be FP64 (global) or FP32 (shared).  The
// staging loops run along whichever index is contiguous in memory.
template <class TC, class TA, class TB>
static __device__ void cta_gemm32(TC* C, int ldc, int m, int n, int kk, double alpha, const TA* A, int lda, bool ta,
                                  const TB* B, int ldb, bool tb, bool zero, float* sm) {
  int tid = threadIdx.x, ti = tid & 15, tj = tid >> 4;
  float* As = sm;                          // KB rows of MB (ld HM_G32_LD)
  float* Bs = sm + HM_G32_KB * HM_G32_LD;  // KB rows of NB (ld HM_G32_LD)
  for (int i0 = 0; i0 < m; i0 += HM_G32_MB) {
    for (int j0 = 0; j0 < n; j0 += HM_G32_NB) {
      float acc[4][4];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
      for (int k0 = 0; k0 < kk; k0 += HM_G32_KB) {
        __syncthreads();
        for (int idx = tid; idx < HM_G32_KB * HM_G32_MB; idx += HM_THREADS) {
          // op(A)(i, l): A[l lda + i] (contiguous in i) or A[i lda + l] (in l)
          int r = ta ? idx / HM_G32_KB : idx % HM_G32_MB, q = ta ? idx % HM_G32_KB : idx / HM_G32_MB;
          int i = i0 + r, l = k0 + q;
          float v = 0.f;
          if (i < m && l < kk) v = (float)(ta ? A[(int64_t)i * lda + l] : A[(int64_t)l * lda + i]);
          As[q * HM_G32_LD + r] = v;
        }
        for (int idx = tid; idx < HM_G32_KB * HM_G32_NB; idx += HM_THREADS) {
          // op(B)(l, j): B[l ldb + j] (contiguous in j) or B[j ldb + l] (in l)
          int c = tb ? idx % HM_G32_NB : idx / HM_G32_KB, q = tb ? idx / HM_G32_NB : idx % HM_G32_KB;
          int j = j0 + c, l = k0 + q;
          float v = 0.f;
          if (j < n && l < kk) v = (float)(tb ? B[(int64_t)l * ldb + j] : B[(int64_t)j * ldb + l]);
          Bs[q * HM_G32_LD + c] = v;
        }
        __syncthreads();
        int kmax = kk - k0 < HM_G32_KB ? kk - k0 : HM_G32_KB;
        for (int q = 0; q < kmax; ++q) {
          float av[4], bv[4];
#pragma unroll
          for (int a = 0; a < 4; ++a) av[a] = As[q * HM_G32_LD + ti * 4 + a];
#pragma unroll
          for (int b = 0; b < 4; ++b) bv[b] = Bs[q * HM_G32_LD + tj * 4 + b];
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] += av[a] * bv[b];
        }
      }
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        int i = i0 + ti * 4 + a;
        if (i >= m) continue;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          int j = j0 + tj * 4 + b;
          if (j >= n) continue;
          TC* c = C + (int64_t)j * ldc + i;
          if constexpr (sizeof(TC) == sizeof(float)) {
            float v = (float)alpha * acc[a][b];
            *c = zero ? v : *c + v;
          } else {
            double v = alpha * (double)acc[a][b];
            *c = zero ? v : *c + v;
          }
        }
      }
    }
  }
  __syncthreads();
}

// floats of s.jac the FP32 work space may use (the rest: the core's W, Vrot,
// norms and permutation, then the staging of cta_gemm32)
#define HM_F32_SMEM ((2 * HM_JAC_SMEM - 6400) & ~127)
// after it: the core's W, Vrot, norms, permutation (2 RMAX^2 + 2 RMAX floats),
// then the staging of cta_gemm32 (HM_G32_SMEM floats), up to the end of s.jac
#define HM_F32_STAGE (HM_F32_SMEM + 2 * HM_RMAX * HM_RMAX + 2 * HM_RMAX)
static_assert(HM_F32_STAGE + HM_G32_SMEM <= 2 * HM_JAC_SMEM, "FP32 scratch exceeds s.jac");

#define HM_F32_MAX_MN (1 << 20)  // largest m n truncated through the FP32 path

static __device__ int trunc_rand32(const float* M, int m, int n, double scale, float* fw, uint32_t* Om, double eps,
                                   int cap, double* U, int ldu, double* V, int ldv, int* status, Smem& s,
                                   double* flops, int* ok, uint64_t seed, int r0) {
  int tid = threadIdx.x;
  if (tid == 0) s.ivals[5] = s.ivals[6] = 0;  // attempts, columns sketched over all attempts
  int rmax = HM_RMAX;
  if (rmax > m) rmax = m;
  if (rmax > n) rmax = n;
  float acc = 0.f;  // per-thread partial sums in FP32, the block sum in FP64
  for (int64_t idx = tid; idx < (int64_t)m * n; idx += HM_THREADS) {
    float x = M[idx];
    acc += x * x;
  }
  double total = block_sum((double)acc, s);
  if (total == 0.0) {
    *ok = 1;
    return 0;
  }
  double bound = eps * eps * total;
  double f = 0.0;
  for (int i = tid; i < n; i += HM_THREADS) Om[i] = (uint32_t)mix64(seed ^ ((uint64_t)i * 0xD1B54A32D192ED03ull));
  int r = r0 < 2 ? 2 : r0;
  if (r > rmax) r = rmax;
  bool fw_shared = __isShared(fw);
  for (;;) {
    __syncthreads();
    if (tid == 0) {
      s.ivals[5] += 1;
      s.ivals[6] += r;
    }
    // this attempt's panels, in shared memory whenever they fit
    float* Y = (!fw_shared && 2 * (int64_t)(m + n) * r <= HM_F32_SMEM) ? (float*)s.jac : fw;  // m x r
    float* Qf = Y + (int64_t)m * r;   // m x r
    float* J = Qf + (int64_t)m * r;   // n x r
    float* Jq = J + (int64_t)n * r;   // n x r: QR of J
    for (int idx = tid; idx < m * r; idx += HM_THREADS) {
      int i = idx % m, j = idx / m;
      float a = 0.f;
      for (int c = 0; c < n; ++c) {
        float x = M[(int64_t)c * m + i];
        a += ((Om[c] >> j) & 1u) ? x : -x;
      }
      Y[(int64_t)j * m + i] = a;
    }
    __syncthreads();
    cta_qr_f(Y, m, m, r, s.tauA, s.rdiagA, s);
    form_q_f(Y, m, m, r, s.tauA, Qf, m, s);
    // J = M^T Q (tiled FP32 product)
    cta_gemm32(J, n, n, r, m, 1.0, M, m, true, Qf, m, false, true, (float*)s.jac + HM_F32_STAGE);
    // sketch, QR and Q of the sketch, J, residual
    count_f32(s, (double)m * n * r + 4.0 * m * r * r + 4.0 * (double)m * n * r);
    float racc = 0.f;
    for (int64_t idx = tid; idx < (int64_t)m * n; idx += HM_THREADS) {
      int i = (int)(idx % m), c = (int)(idx / m);
      float a = M[idx];
      for (int j = 0; j < r; ++j) a -= Qf[(int64_t)j * m + i] * J[(int64_t)j * n + c];
      racc += a * a;
    }
    double res2 = block_sum((double)racc, s);
    if (!(res2 <= bound)) {  // also catches a non-finite residual
      if (r >= rmax || !isfinite(res2)) {
        *ok = 0;
        return 0;
      }
      r = 2 * r > rmax ? rmax : 2 * r;
      continue;
    }
    // Core: column-pivoted QR of J, a few Jacobi sweeps on R^T (core_f32);
    // J itself becomes Q_J explicitly afterwards.
    for (int idx = tid; idx < n * r; idx += HM_THREADS) Jq[idx] = J[idx];
    __syncthreads();
    float* cw = (float*)(s.jac + HM_F32_SMEM / 2);  // 2 r^2 + 2 r floats
    core_f32(Jq, n, r, cw, s, HM_CORE_SWEEPS);
    form_q_f(Jq, n, n, r, s.tauB, J, n, s);
    // pivoted QR, Q_J, rotations (12 r per rotation: dots and updates)
    count_f32(s, 4.0 * n * r * r + 12.0 * r * (double)s.ivals[3]);
    if (tid == 0) {
      double tail = res2;
      int k = r;
      while (k > 0) {
        double x = s.sigma[s.order[k - 1]];
        if (tail + x * x <= bound) {
          tail += x * x;
          --k;
        } else {
          break;
        }
      }
      s.ivals[4] = k;
    }
    __syncthreads();
    int k = s.ivals[4];
    __syncthreads();
    if (k > cap) {
      if (tid == 0) set_status(status, DS_RANK);
      k = cap;
    }
    if (k > 0) {
      // M ~ (Q P W_k)(Q_J Vrot_k)^T = (Q P Wh)(Q_J Z)^T: C = Q P Wh, D = Q_J Z
      // (Y and Jq are free: the sketch's and J's reflectors have been used)
      core_f32_orth(cw, r, k, Y, Jq, s);
      count_f32(s, 4.0 * r * k * k + 2.0 * (m + n) * (double)r * k);
      const float* Wh = Jq;
      const float* Z = cw;
      const int* perm = (const int*)(cw + 2 * r * r + r);
      for (int idx = tid; idx < m * k; idx += HM_THREADS) {
        int i = idx % m, jj = idx / m;
        const float* wc = Wh + (int64_t)jj * r;
        float a = 0.f;
        for (int j = 0; j < r; ++j) a += Qf[(int64_t)perm[j] * m + i] * wc[j];
        U[(int64_t)jj * ldu + i] = (double)a;
      }
      for (int idx = tid; idx < n * k; idx += HM_THREADS) {
        int c = idx % n, jj = idx / n;
        const float* zc = Z + (int64_t)jj * r;
        float a = 0.f;
        for (int j = 0; j < r; ++j) a += J[(int64_t)j * n + c] * zc[j];
        V[(int64_t)jj * ldv + c] = (double)a * scale;
      }
    }
    if (flops && tid == 0) *flops += f;
    *ok = 1;
    return k;
  }
}

#define HM_FACT32_DIRECT 64  // largest stacked width truncated without a sketch
static_assert(2 * HM_FACT32_DIRECT * HM_FACT32_DIRECT + 2 * HM_FACT32_DIRECT <= 2 * HM_JAC_SMEM,
              "direct FP32 core exceeds s.jac");
// ---------------------------------------------------------------------------
// Mixed-precision truncation of a factored M = SA SB^T (m x n, stacked width
// l <= min(m, n)), the steps of Fig. rkadd in FP32: SB = Q_B R_B (Householder), then
// Mhat = SA R_B^T (m x l) carries all of M (M = Mhat Q_B^T, Q_B orthonormal),
// so truncating Mhat by trunc_rand32 truncates M with the same error, and
// D = Q_B Dhat.  SAf, SBf: FP32 copies scaled so that |SAf SBf^T| <= 1
// entrywise (scale S restores M).  Mhat is formed with the cancellation guard
// of the explicit path (a failure returns with *ok = 0, *guard = 1).
// Float scratch fs: Mhat (m l), Q_B (n l), panels 2 (m + l) RMAX, l sign
// words; double scratch ds: 2 l + l RMAX.
// ---------------------------------------------------------------------------
static __device__ int trunc_fact32(int m, int n, int l, const float* SAf, float* SBf, double S, float* fs,
                                   double* ds, double eps, int cap, double* U, int ldu, double* V, int ldv,
                                   int* status, Smem& s, double* flops, int* ok, int* guard, uint64_t seed, int r0) {
  int tid = threadIdx.x;
  *ok = 0;
  *guard = 0;
  float* Mh = fs;
  float* QB = Mh + (int64_t)m * l;
  float* pan = QB + (int64_t)n * l;
  uint32_t* Om = (uint32_t*)(pan + 2 * (int64_t)(m + l) * HM_RMAX);
  double* tq = ds;
  double* rq = ds + l;
  double* Vh = ds + 2 * l;  // l x k (ld l)
  cta_qr_f(SBf, n, n, l, tq, rq, s);
  count_f32(s, 2.0 * n * l * l + (double)m * l * l);  // QR of SB, Mhat
  float sm = 0.f, sabs = 0.f;
  for (int idx = tid; idx < m * l; idx += HM_THREADS) {
    int i = idx % m, c = idx / m;
    float v = 0.f, a = 0.f;
    for (int j = c; j < l; ++j) {
      float rcj = j == c ? (float)rq[c] : SBf[(int64_t)j * n + c];
      float x = SAf[(int64_t)j * m + i] * rcj;
      v += x;
      a += fabsf(x);
    }
    Mh[idx] = v;
    sm += v * v;
    sabs += a * a;
  }
  double tm = block_sum((double)sm, s), ta = block_sum((double)sabs, s);
  if (!isfinite(tm) || !isfinite(ta) || ta * 9e-14 > 1e-2 * eps * eps * tm) {
    *guard = 1;
    return 0;
  }
  if (l <= HM_FACT32_DIRECT && l <= m) {
    // Mhat has at most l <= 64 columns (and at least as many rows, so that its
    // R factor is l x l): its pivoted QR and a few Jacobi sweeps
    // (core_f32) are the whole truncation, Mhat = (Q_J Vrot)(P W)^T, so
    // C = Q_J Vrot(:, order) and D = Q_B P W(:, order) S, with no sketch
    // (and no sketch that could miss).  s.jac is free here: the core's W,
    // Vrot, norms and permutation sit at its start.
    if (tid == 0) s.ivals[5] = s.ivals[6] = 0;
    float* cw = (float*)s.jac;
    core_f32(Mh, m, l, cw, s, HM_CORE_SWEEPS);
    if (tid == 0) {
      double total = 0.0;
      for (int i = 0; i < l; ++i) total += s.sigma[i] * s.sigma[i];
      double bound = eps * eps * total, tail = 0.0;
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
      if (k > cap) {
        set_status(status, DS_RANK);
        k = cap;
      }
      s.ivals[4] = k;
    }
    __syncthreads();
    int k = s.ivals[4];
    // C = Q_J [Vrot(:, order); 0] and D = Q_B [P W(:, order); 0] S: the
    // reflectors applied to the k kept columns (m x k in pan, n x k in QB)
    const float* W = cw;
    const float* Vrot = cw + l * l;
    const int* perm = (const int*)(cw + 2 * l * l + l);
    float* Cf = (float*)SAf;  // SAf is dead once Mhat is formed
    float* Df = QB;
    for (int idx = tid; idx < m * k; idx += HM_THREADS) {
      int i = idx % m, jj = idx / m;
      Cf[idx] = i < l ? Vrot[(int64_t)s.order[jj] * l + i] : 0.f;
    }
    for (int idx = tid; idx < n * k; idx += HM_THREADS) Df[idx] = 0.f;
    __syncthreads();
    for (int idx = tid; idx < l * k; idx += HM_THREADS) {
      int j = idx % l, jj = idx / l;
      Df[(int64_t)jj * n + perm[j]] = W[(int64_t)s.order[jj] * l + j];
    }
    cta_apply_qf(Mh, m, m, l, s.tauB, Cf, m, k, s);
    cta_apply_qf(SBf, n, n, l, tq, Df, n, k, s);
    for (int idx = tid; idx < m * k; idx += HM_THREADS) U[(int64_t)(idx / m) * ldu + idx % m] = (double)Cf[idx];
    for (int idx = tid; idx < n * k; idx += HM_THREADS) V[(int64_t)(idx / n) * ldv + idx % n] = (double)Df[idx] * S;
    count_f32(s, 2.0 * m * l * l + 12.0 * l * (double)s.ivals[3] + 4.0 * (m + n) * (double)l * k);
    __syncthreads();
    *ok = 1;
    return k;
  }
  int k = trunc_rand32(Mh, m, l, S, pan, Om, eps, cap, U, ldu, Vh, l, status, s, flops, ok, seed, r0);
  if (!*ok) return 0;
  form_q_f(SBf, n, n, l, tq, QB, n, s);
  count_f32(s, 2.0 * n * l * l + 2.0 * n * (double)l * k);  // Q_B, D = Q_B Dhat
  for (int idx = tid; idx < n * k; idx += HM_THREADS) {
    int c = idx % n, jj = idx / n;
    float a = 0.f;
    for (int j = 0; j < l; ++j) a += QB[(int64_t)j * n + c] * (float)Vh[(int64_t)jj * l + j];
    V[(int64_t)jj * ldv + c] = (double)a;
  }
  __syncthreads();
  return k;
}

// Scratch of trunc_fact32 past the FP32 factor copies: floats, then doubles.
__host__ __device__ inline int64_t fact32_floats(int64_t m, int64_t n, int64_t l) {
  return m * l + n * l + 2 * (m + l) * HM_RMAX + l + 2;
}

// FP32 factored truncation of M = SA [blockdiag(SB0, SB1)]^T (m x n, n = n0 +
// n1, l = k0 + k1 <= min(m, n); SB1 may be null): the factors are copied to
// FP32, each scaled by its largest entry, then trunc_fact32.  ws: the float
// copies and trunc_fact32's scratch (or shared memory, for the direct path
// when it all fits).  Returns the rank; *ok = 0 when the caller must fall
// back to the exact truncation; *S_out = the scale of M.
static __device__ int fact32_run(int m, int n, int l, const double* SA, const double* SB0, int n0, int k0,
                                 const double* SB1, int n1, int k1, double* ws, double eps, int cap, double* U, int ldu,
                                 double* V, int ldv, int* status, Smem& s, uint64_t seed, int r0, double* f, int* ok,
                                 double* S_out) {
  int tid = threadIdx.x;
  *ok = 0;
  *S_out = 0.0;
  double ma = 0.0, mb = 0.0;
  for (int idx = tid; idx < m * l; idx += HM_THREADS) ma = fmax(ma, fabs(SA[idx]));
  for (int idx = tid; idx < n0 * k0; idx += HM_THREADS) mb = fmax(mb, fabs(SB0[idx]));
  for (int idx = tid; idx < n1 * k1; idx += HM_THREADS) mb = fmax(mb, fabs(SB1[idx]));
  ma = block_max(ma, s);
  mb = block_max(mb, s);
  double S = ma * mb;
  *S_out = S;
  if (!(S > 0.0) || !isfinite(S)) return 0;
  float* SAf = (float*)ws;
  float* SBf = SAf + (int64_t)m * l;
  float* fs = SBf + (int64_t)n * l;
  int64_t nf = (int64_t)m * l + (int64_t)n * l + fact32_floats(m, n, l);
  double* ds = ws + (nf + 1) / 2;
  // The direct path (no sketch) with everything in shared memory when it
  // fits: the core's W, Vrot, norms and permutation at the start of s.jac,
  // then SAf (later C), SBf, Mhat, Q_B's columns (later D), the QR's tau and
  // R diagonal.
  int64_t cwsz = (2 * (int64_t)l * l + 2 * l + 3) & ~(int64_t)3;
  int64_t panel = 2 * (int64_t)(m + n) * l;
  if (l <= HM_FACT32_DIRECT && l <= m && cwsz + panel + 4 * l + 8 <= 2 * (int64_t)HM_JAC_SMEM) {
    SAf = (float*)s.jac + cwsz;
    SBf = SAf + (int64_t)m * l;
    fs = SBf + (int64_t)n * l;
    ds = (double*)(((uintptr_t)(fs + (int64_t)(m + n) * l) + 7) & ~(uintptr_t)7);
  }
  double ia = 1.0 / ma, ib = 1.0 / mb;
  for (int idx = tid; idx < m * l; idx += HM_THREADS) SAf[idx] = (float)(SA[idx] * ia);
  for (int idx = tid; idx < n * l; idx += HM_THREADS) {
    int c = idx % n, j = idx / n;
    double v = 0.0;
    if (j < k0) {
      if (c < n0) v = SB0[(int64_t)j * n0 + c];
    } else if (c >= n0) {
      v = SB1[(int64_t)(j - k0) * n1 + (c - n0)];
    }
    SBf[idx] = (float)(v * ib);
  }
  __syncthreads();
  int guard = 0;
  return trunc_fact32(m, n, l, SAf, SBf, S, fs, ds, eps, cap, U, ldu, V, ldv, status, s, f, ok, &guard, seed, r0);
}

// Doubles of scratch trunc_rand needs.
__host__ __device__ inline int64_t rand_ws_doubles(int64_t m, int64_t n, int64_t l) {
  int64_t g = 2 * l * l;
  if (g < l * HM_RMAX) g = l * HM_RMAX;
  return 2 * m * HM_RMAX + n * HM_RMAX + HM_RMAX * HM_RMAX + (n + 1) / 2 + 1 + g +
         (2 * n * HM_RMAX + 4 * HM_RMAX * HM_RMAX + 2 * HM_RMAX + 1) / 2 + 64;
}

// ---------------------------------------------------------------------------
// Dense leaf operations
// ---------------------------------------------------------------------------
// No-pivot LU in place (L unit lower, U upper).
static __device__ void cta_lu(double* A, int ld, int n, int* status) {
  int tid = threadIdx.x;
  for (int k = 0; k < n; ++k) {
    double piv = A[(int64_t)k * ld + k];
    if (piv == 0.0 || !isfinite(piv)) {
      if (tid == 0) set_status(status, piv == 0.0 ? DS_SINGULAR : DS_NONFINITE);
      return;
    }
    double inv = 1.0 / piv;
    for (int i = k + 1 + tid; i < n; i += HM_THREADS) A[(int64_t)k * ld + i] *= inv;
    __syncthreads();
    int rem = n - k - 1;
    for (int idx = tid; idx < rem * rem; idx += HM_THREADS) {
      int i = k + 1 + idx % rem, j = k + 1 + idx / rem;
      A[(int64_t)j * ld + i] -= A[(int64_t)k * ld + i] * A[(int64_t)j * ld + k];
    }
    __syncthreads();
  }
}

// Thin solves with a dense diagonal leaf N (n x n, ld): X (n x w, ldx).
// One warp per right-hand-side column: columns are independent, so the
// substitution needs only warp-level synchronisation.
template <class T>
static __device__ void cta_trsm_cols_t(int kind, const T* N, int ld, int n, T* X, int ldx, int w) {
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int c = warp; c < w; c += HM_WARPS) {
    T* x = X + (int64_t)c * ldx;
    if (kind == TRSM_L) {
      for (int k = 0; k < n - 1; ++k) {
        T xk = x[k];
        for (int i = k + 1 + lane; i < n; i += 32) x[i] -= N[(int64_t)k * ld + i] * xk;
        __syncwarp();
      }
    } else if (kind == TRSM_U) {
      for (int k = n - 1; k >= 0; --k) {
        T xk = x[k] / N[(int64_t)k * ld + k];
        __syncwarp();
        if (lane == 0) x[k] = xk;
        for (int i = lane; i < k; i += 32) x[i] -= N[(int64_t)k * ld + i] * xk;
        __syncwarp();
      }
    } else if (kind == TRSM_UT) {
      for (int k = 0; k < n; ++k) {
        T xk = x[k] / N[(int64_t)k * ld + k];
        __syncwarp();
        if (lane == 0) x[k] = xk;
        for (int i = k + 1 + lane; i < n; i += 32) x[i] -= N[(int64_t)i * ld + k] * xk;
        __syncwarp();
      }
    } else {
      for (int k = n - 1; k > 0; --k) {
        T xk = x[k];
        for (int i = lane; i < k; i += 32) x[i] -= N[(int64_t)i * ld + k] * xk;
        __syncwarp();
      }
    }
  }
  __syncthreads();
}
static __device__ void cta_trsm_cols(int kind, const double* N, int ld, int n, double* X, int ldx, int w) {
  cta_trsm_cols_t<double>(kind, N, ld, n, X, ldx, w);
}

// Thin triangular solve: the triangle and the right-hand sides are staged in
// shared memory when they fit (coalesced loads, then the warp substitutions
// run on shared memory), else solved in place in global memory.
static __device__ void cta_trsm(int kind, const double* N, int ld, int n, double* X, int ldx, int w, Smem& s) {
  if (w <= 0) return;
  if ((int64_t)n * n + (int64_t)n * w <= HM_JAC_SMEM) {
    double* Ns = s.jac;
    double* Xs = s.jac + (int64_t)n * n;
    for (int idx = threadIdx.x; idx < n * n; idx += HM_THREADS) Ns[idx] = N[(int64_t)(idx / n) * ld + idx % n];
    for (int idx = threadIdx.x; idx < n * w; idx += HM_THREADS) Xs[idx] = X[(int64_t)(idx / n) * ldx + idx % n];
    __syncthreads();
    cta_trsm_cols(kind, Ns, n, n, Xs, n, w);
    for (int idx = threadIdx.x; idx < n * w; idx += HM_THREADS) X[(int64_t)(idx / n) * ldx + idx % n] = Xs[idx];
    __syncthreads();
  } else {
    cta_trsm_cols(kind, N, ld, n, X, ldx, w);
  }
}

// C (m x n, ldc) (+)= alpha op(A) op(B), op(A) m x kk, op(B) kk x n.
static __device__ void cta_gemm(double* C, int ldc, int m, int n, int kk, double alpha, const double* A, int lda,
                         bool ta, const double* B, int ldb, bool tb, bool zero) {
  int tid = threadIdx.x;
  for (int idx = tid; idx < m * n; idx += HM_THREADS) {
    int i = idx % m, j = idx / m;
    double acc = 0.0;
    for (int l = 0; l < kk; ++l) {
      double a = ta ? A[(int64_t)i * lda + l] : A[(int64_t)l * lda + i];
      double b = tb ? B[(int64_t)l * ldb + j] : B[(int64_t)j * ldb + l];
      acc += a * b;
    }
    double* c = C + (int64_t)j * ldc + i;
    *c = zero ? alpha * acc : *c + alpha * acc;
  }
}

// ---------------------------------------------------------------------------
// FP32 leaf operations of the mixed path (eps >= HM_F32_MIN_EPS): operands
// are staged once as FP32 in shared memory, products and sums run in FP32,
// results are stored back in FP64.
// ---------------------------------------------------------------------------
// cta_trsm in FP32; returns false (nothing done) if N and X do not fit.
static __device__ bool cta_trsm_f32(int kind, const double* N, int ld, int n, double* X, int ldx, int w, Smem& s) {
  if (w <= 0) return true;
  if ((int64_t)n * n + (int64_t)n * w > 2 * HM_JAC_SMEM) return false;
  float* Ns = (float*)s.jac;
  float* Xs = Ns + (int64_t)n * n;
  for (int idx = threadIdx.x; idx < n * n; idx += HM_THREADS) Ns[idx] = (float)N[(int64_t)(idx / n) * ld + idx % n];
  for (int idx = threadIdx.x; idx < n * w; idx += HM_THREADS) Xs[idx] = (float)X[(int64_t)(idx / n) * ldx + idx % n];
  __syncthreads();
  cta_trsm_cols_t<float>(kind, Ns, n, n, Xs, n, w);
  count_f32(s, (double)n * n * w);
  for (int idx = threadIdx.x; idx < n * w; idx += HM_THREADS) X[(int64_t)(idx / n) * ldx + idx % n] = (double)Xs[idx];
  __syncthreads();
  return true;
}

}  // namespace hm
