// hmat_oracle.cpp -- CPU oracle for H-matrix arithmetic with accumulated updates.
//
// TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, serial FP64
// statement of what the hot path computes (Boerm, "Hierarchical matrix
// arithmetic with accumulated updates", arXiv:1703.09085).  Only tests/,
// __graft_entry__.smoke() and bench.py's cpu_baseline / reference arm may load
// it.  It shares no code with the CUDA path in paper_1703_09085_gb300/.
//
// Every procedure follows the paper's figure or paragraph named in its
// comment, in the paper's order of steps.  Dense building blocks are
// textbook: Householder QR (Golub & Van Loan, Matrix Computations, Alg. 5.2.1),
// one-sided Jacobi SVD (Hestenes 1958; Demmel & Veselic 1992), no-pivot
// Gaussian elimination.  No blocking, fusion or reordering beyond that.
//
// Readings where the paper is silent or inconsistent:
//  * cluster tree: geometric bisection at the midpoint of the tight bounding
//    box along its longest side (first side on ties), stable partition
//    "coordinate < midpoint" -> first son; the paper only requires a cluster
//    tree (Section 2, Definition "Cluster tree") and a binary one in Section 6.
//  * admissibility: (t,s) is an admissible leaf iff dist(t,s) > 0 and
//    max(diam t, diam s) <= eta * dist(t,s), with diam the Euclidean diagonal
//    of the tight box and dist the Euclidean box distance.
//  * "Choose new rank k" (Fig. rkadd, Fig. rowmerge): smallest k with
//    sum_{i>k} sigma_i^2 <= eps^2 * sum_i sigma_i^2 (relative Frobenius, per
//    block); eps = 0 keeps every nonzero singular value.
//  * Fig. addevaltrans, inadmissible case: read as X <- X + alpha N_b^* Y.
//  * Fig. addproduct, second case with #r <= #s: alpha is applied once, in
//    rkadd; addeval uses 1 as in the other three cases.
//  * Fig. rkupdate, inadmissible case: N_b <- N_b + alpha A B^*.
//  * Fig. flush: the recursive call on the sons uses Z restricted to t' x r'.
//  * A product whose low-rank form has zero columns is the zero matrix and
//    is not added (no truncation is run for it).
//  * H-LU with accumulators: the paper only says LR and Cholesky are "treated
//    in a similar way" as the inversion of Fig. invert (Section 6).  The
//    recursion used here is the block LU with Schur complement
//    G22 - G21 G11^{-1} G12 of Section 6, with the accumulator split as in
//    Fig. invert: lu(t1); flush + solve the off-diagonal blocks; addproduct
//    the Schur update without flush; lu(t2) takes the accumulator.
//  * Fig. invert: its last product, H_12 H_21', is accumulated for the block
//    t_1 x t_1 and flushed into G_11 (the figure's index t_2 there is read as
//    t_1, the block H_11' overwrites); a flushed accumulator is not reused.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

namespace orc {

typedef int64_t i64;

// ---------------------------------------------------------------------------
// Statistics (what the method did, for tests and the CPU baseline)
// ---------------------------------------------------------------------------
struct Stats {
  i64 truncations;   // rank-revealing factorisations: rkadd + rowmerge SVDs
  i64 rkadds;
  i64 rowmerges;
  i64 addproducts;   // calls of Fig. addproduct that evaluated a product
  i64 pending;       // calls of Fig. addproduct that appended a pending product
  i64 dense_lu;
  double flops;      // counted floating-point operations (estimate)
  double seconds;
  double flops_trunc;  // of which inside truncations (QR, SVD, factor products)
  double flops_dense;  // of which in dense leaf LU / triangular solves
};
static Stats g_stats;
// Optional record of every truncation: rows, columns, stacked width, new rank.
static bool g_trace_on = false;
static std::vector<int64_t> g_trace;
static void trace_trunc(int64_t m, int64_t n, int64_t l, int64_t k) {
  if (!g_trace_on) return;
  g_trace.push_back(m);
  g_trace.push_back(n);
  g_trace.push_back(l);
  g_trace.push_back(k);
}
static int g_cat = 0;  // 0 products and updates, 1 truncation, 2 dense leaf
static void count_flops(double f) {
  g_stats.flops += f;
  if (g_cat == 1) g_stats.flops_trunc += f;
  if (g_cat == 2) g_stats.flops_dense += f;
}
struct CatScope {
  int saved;
  explicit CatScope(int c) : saved(g_cat) { g_cat = c; }
  ~CatScope() { g_cat = saved; }
};

struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};
enum { OK = 0, ERR_ARG = 1, ERR_SINGULAR = 3, ERR_INTERNAL = 9 };

// ---------------------------------------------------------------------------
// Dense column-major matrices
// ---------------------------------------------------------------------------
struct Mat {
  i64 m = 0, n = 0;
  std::vector<double> a;
  Mat() {}
  Mat(i64 m_, i64 n_) : m(m_), n(n_), a((size_t)(m_ * n_), 0.0) {}
#ifdef ORC_BOUNDS
  double& operator()(i64 i, i64 j) {
    if (i < 0 || i >= m || j < 0 || j >= n) throw Error(ERR_INTERNAL, "Mat index out of range");
    return a[(size_t)(i + j * m)];
  }
  double operator()(i64 i, i64 j) const {
    if (i < 0 || i >= m || j < 0 || j >= n) throw Error(ERR_INTERNAL, "Mat index out of range");
    return a[(size_t)(i + j * m)];
  }
#else
  double& operator()(i64 i, i64 j) { return a[(size_t)(i + j * m)]; }
  double operator()(i64 i, i64 j) const { return a[(size_t)(i + j * m)]; }
#endif
};

static Mat identity(i64 n) {
  Mat I(n, n);
  for (i64 i = 0; i < n; ++i) I(i, i) = 1.0;
  return I;
}

static Mat transpose(const Mat& A) {
  Mat T(A.n, A.m);
  for (i64 j = 0; j < A.n; ++j)
    for (i64 i = 0; i < A.m; ++i) T(j, i) = A(i, j);
  return T;
}

// Rows [r0, r0+cnt) of A.
static Mat rows_of(const Mat& A, i64 r0, i64 cnt) {
  Mat R(cnt, A.n);
  for (i64 j = 0; j < A.n; ++j)
    for (i64 i = 0; i < cnt; ++i) R(i, j) = A(r0 + i, j);
  return R;
}

static void set_rows(Mat& A, i64 r0, const Mat& R) {
  for (i64 j = 0; j < A.n; ++j)
    for (i64 i = 0; i < R.m; ++i) A(r0 + i, j) = R(i, j);
}

// [A B] (same number of rows).
static Mat hcat(const Mat& A, const Mat& B) {
  i64 m = A.n ? A.m : B.m;
  Mat C(m, A.n + B.n);
  for (i64 j = 0; j < A.n; ++j)
    for (i64 i = 0; i < m; ++i) C(i, j) = A(i, j);
  for (i64 j = 0; j < B.n; ++j)
    for (i64 i = 0; i < m; ++i) C(i, A.n + j) = B(i, j);
  return C;
}

// C(rows c0.., :) += alpha * op(A) * op(B).  op(X) = X or X^T.
static void gemm_acc(bool ta, bool tb, double alpha, const Mat& A, const Mat& B, Mat& C,
                     i64 c0 = 0) {
  i64 m = ta ? A.n : A.m;
  i64 k = ta ? A.m : A.n;
  i64 n = tb ? B.m : B.n;
  i64 kb = tb ? B.n : B.m;
  if (k != kb || c0 + m > C.m || n != C.n) throw Error(ERR_INTERNAL, "gemm: shape mismatch");
  count_flops(2.0 * (double)m * (double)n * (double)k);
  for (i64 j = 0; j < n; ++j) {
    for (i64 l = 0; l < k; ++l) {
      double b = tb ? B(j, l) : B(l, j);
      if (b == 0.0) continue;
      double ab = alpha * b;
      if (!ta) {
        const double* acol = &A.a[(size_t)(l * A.m)];
        double* ccol = &C.a[(size_t)(c0 + j * C.m)];
        for (i64 i = 0; i < m; ++i) ccol[i] += ab * acol[i];
      } else {
        for (i64 i = 0; i < m; ++i) C(c0 + i, j) += ab * A(l, i);
      }
    }
  }
}

static Mat matmul(bool ta, bool tb, const Mat& A, const Mat& B) {
  Mat C(ta ? A.n : A.m, tb ? B.m : B.n);
  gemm_acc(ta, tb, 1.0, A, B, C);
  return C;
}

// ---------------------------------------------------------------------------
// Householder QR, Golub & Van Loan Alg. 5.2.1 (thin form).
// A (m x n) = Q R with Q (m x q) orthonormal columns, R (q x n) upper
// trapezoidal, q = min(m, n).
// ---------------------------------------------------------------------------
static void householder_qr(const Mat& A, Mat& Q, Mat& R) {
  i64 m = A.m, n = A.n, q = std::min(m, n);
  Mat W = A;
  std::vector<std::vector<double>> vs((size_t)q);
  std::vector<double> betas((size_t)q, 0.0);
  for (i64 j = 0; j < q; ++j) {
    // Reflector P = I - beta v v^T with P x = alpha e1 for x = W(j:m, j).
    // P does not change when v is scaled, so v is built from x / max|x_i|
    // to keep the squared norms clear of underflow and overflow.
    std::vector<double> v((size_t)(m - j));
    double scale = 0.0;
    for (i64 i = j; i < m; ++i) scale = std::max(scale, std::fabs(W(i, j)));
    double beta = 0.0;
    if (scale > 0.0) {
      double xnorm2 = 0.0;
      for (i64 i = j; i < m; ++i) {
        v[(size_t)(i - j)] = W(i, j) / scale;
        xnorm2 += v[(size_t)(i - j)] * v[(size_t)(i - j)];
      }
      double xnorm = std::sqrt(xnorm2);
      double alpha = (v[0] >= 0.0) ? -xnorm : xnorm;
      v[0] -= alpha;
      double vnorm2 = 0.0;
      for (double x : v) vnorm2 += x * x;
      beta = 2.0 / vnorm2;
    }
    // Apply to the trailing columns j..n-1.
    for (i64 c = j; c < n; ++c) {
      double d = 0.0;
      for (i64 i = j; i < m; ++i) d += v[(size_t)(i - j)] * W(i, c);
      d *= beta;
      for (i64 i = j; i < m; ++i) W(i, c) -= d * v[(size_t)(i - j)];
    }
    vs[(size_t)j] = std::move(v);
    betas[(size_t)j] = beta;
  }
  count_flops(4.0 * (double)m * (double)n * (double)q);
  R = Mat(q, n);
  for (i64 j = 0; j < n; ++j)
    for (i64 i = 0; i <= std::min(j, q - 1); ++i) R(i, j) = W(i, j);
  // Backward accumulation of the thin Q = P_0 ... P_{q-1} I(:, 0:q).
  Q = Mat(m, q);
  for (i64 i = 0; i < q; ++i) Q(i, i) = 1.0;
  for (i64 j = q - 1; j >= 0; --j) {
    const std::vector<double>& v = vs[(size_t)j];
    for (i64 c = j; c < q; ++c) {
      double d = 0.0;
      for (i64 i = j; i < m; ++i) d += v[(size_t)(i - j)] * Q(i, c);
      d *= betas[(size_t)j];
      for (i64 i = j; i < m; ++i) Q(i, c) -= d * v[(size_t)(i - j)];
    }
  }
}

// ---------------------------------------------------------------------------
// One-sided Jacobi SVD (Hestenes; Demmel & Veselic) of a p x q matrix with
// p >= q: rotate column pairs until all are mutually orthogonal.
// Returns U (p x q), s (q, descending), V (q x q) with M = U diag(s) V^T.
// ---------------------------------------------------------------------------
static void jacobi_svd_tall(const Mat& M, Mat& U, std::vector<double>& s, Mat& V) {
  i64 p = M.m, q = M.n;
  Mat W = M;
  V = identity(q);
  const double tol = 1e-15;
  for (int sweep = 0; sweep < 80; ++sweep) {
    bool rotated = false;
    for (i64 i = 0; i < q - 1; ++i) {
      for (i64 j = i + 1; j < q; ++j) {
        double alpha = 0.0, beta = 0.0, gamma = 0.0;
        for (i64 r = 0; r < p; ++r) {
          alpha += W(r, i) * W(r, i);
          beta += W(r, j) * W(r, j);
          gamma += W(r, i) * W(r, j);
        }
        count_flops(6.0 * (double)p);
        if (alpha == 0.0 || beta == 0.0) continue;
        if (std::fabs(gamma) <= tol * std::sqrt(alpha) * std::sqrt(beta)) continue;
        rotated = true;
        double zeta = (beta - alpha) / (2.0 * gamma);
        double t = (zeta >= 0.0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        double c = 1.0 / std::sqrt(1.0 + t * t);
        double sn = c * t;
        for (i64 r = 0; r < p; ++r) {
          double wi = W(r, i), wj = W(r, j);
          W(r, i) = c * wi - sn * wj;
          W(r, j) = sn * wi + c * wj;
        }
        for (i64 r = 0; r < q; ++r) {
          double vi = V(r, i), vj = V(r, j);
          V(r, i) = c * vi - sn * vj;
          V(r, j) = sn * vi + c * vj;
        }
        count_flops(6.0 * (double)(p + q));
      }
    }
    if (!rotated) break;
  }
  std::vector<double> norms((size_t)q);
  for (i64 j = 0; j < q; ++j) {
    double x = 0.0;
    for (i64 r = 0; r < p; ++r) x += W(r, j) * W(r, j);
    norms[(size_t)j] = std::sqrt(x);
  }
  std::vector<i64> order((size_t)q);
  for (i64 j = 0; j < q; ++j) order[(size_t)j] = j;
  std::stable_sort(order.begin(), order.end(),
                   [&](i64 a, i64 b) { return norms[(size_t)a] > norms[(size_t)b]; });
  U = Mat(p, q);
  Mat Vs(q, q);
  s.assign((size_t)q, 0.0);
  for (i64 jj = 0; jj < q; ++jj) {
    i64 j = order[(size_t)jj];
    double nj = norms[(size_t)j];
    s[(size_t)jj] = nj;
    for (i64 r = 0; r < p; ++r) U(r, jj) = nj > 0.0 ? W(r, j) / nj : 0.0;
    for (i64 r = 0; r < q; ++r) Vs(r, jj) = V(r, j);
  }
  V = Vs;
}

// Thin SVD of an m x q matrix: M = U diag(s) V^T, U (m x p), V (q x p),
// p = min(m, q).  Tall matrices are reduced by Householder QR first, wide
// ones are handled through their transpose.
static void svd_thin(const Mat& M, Mat& U, std::vector<double>& s, Mat& V) {
  if (M.m >= M.n) {
    Mat Q, R;
    householder_qr(M, Q, R);  // R is q x q
    Mat Ur;
    jacobi_svd_tall(R, Ur, s, V);
    U = matmul(false, false, Q, Ur);
  } else {
    Mat T = transpose(M);
    Mat Q, R;
    householder_qr(T, Q, R);
    Mat Ur, Vr;
    jacobi_svd_tall(R, Ur, s, Vr);
    // M^T = (Q Ur) S Vr^T  =>  M = Vr S (Q Ur)^T
    U = Vr;
    V = matmul(false, false, Q, Ur);
  }
}

// Rank rule of "choose new rank k": 0 relative Frobenius (the default), 1
// relative spectral (smallest k with s_{k+1} <= eps s_1).  Set for a call by
// orc_set_rank_rule.
static int g_rank_rule = 0;

// "Choose new rank k" (Fig. rkadd / Fig. rowmerge): smallest k with
// sum_{i>k} s_i^2 <= eps^2 sum_i s_i^2 (or, under the spectral rule, the
// number of s_i > eps s_1), optionally capped at max_rank.  s is in
// decreasing order.
static i64 choose_rank(const std::vector<double>& s, double eps, i64 max_rank) {
  if (g_rank_rule == 1) {
    i64 k = 0;
    double s1 = s.empty() ? 0.0 : s[0];
    while (k < (i64)s.size() && s[(size_t)k] > eps * s1) ++k;
    if (max_rank >= 0 && k > max_rank) k = max_rank;
    return k;
  }
  double total = 0.0;
  for (double x : s) total += x * x;
  i64 k = (i64)s.size();
  double tail = 0.0;
  double bound = eps * eps * total;
  while (k > 0) {
    double x = s[(size_t)(k - 1)];
    if (tail + x * x <= bound) {
      tail += x * x;
      --k;
    } else {
      break;
    }
  }
  if (max_rank >= 0 && k > max_rank) k = max_rank;
  return k;
}

// ---------------------------------------------------------------------------
// Low-rank matrices R = A B^T and truncation (Section 3, "Truncation").
// ---------------------------------------------------------------------------
struct LowRank {
  Mat A, B;  // A: rows x k, B: cols x k
  i64 k() const { return A.n; }
};

struct TruncOpts {
  double eps = 0.0;
  i64 max_rank = -1;
};

// Best rank-k approximation of A B^T (Section 3, "Truncation"): thin QR
// B = Q_B R_B, Ahat = A R_B^T, thin SVD Ahat = U S Vhat^T, then
// C = U(:,1:k), D = Q_B Vhat(:,1:k) S(1:k,1:k)  (as in Fig. rkadd).
static LowRank truncate(const Mat& A, const Mat& B, const TruncOpts& o) {
  CatScope cat(1);
  LowRank out;
  i64 m = A.m, n = B.m;
  if (A.n == 0) {
    out.A = Mat(m, 0);
    out.B = Mat(n, 0);
    return out;
  }
  g_stats.truncations++;
  Mat QB, RB;
  householder_qr(B, QB, RB);                 // QB: n x q, RB: q x l
  Mat Ahat = matmul(false, true, A, RB);     // m x q
  Mat U, Vh;
  std::vector<double> s;
  svd_thin(Ahat, U, s, Vh);                  // U: m x p, Vh: q x p
  i64 k = choose_rank(s, o.eps, o.max_rank);
  trace_trunc(m, n, A.n, k);
  out.A = Mat(m, k);
  for (i64 j = 0; j < k; ++j)
    for (i64 i = 0; i < m; ++i) out.A(i, j) = U(i, j);
  Mat VS(Vh.m, k);
  for (i64 j = 0; j < k; ++j)
    for (i64 i = 0; i < Vh.m; ++i) VS(i, j) = Vh(i, j) * s[(size_t)j];
  out.B = matmul(false, false, QB, VS);      // n x k
#ifdef ORC_BOUNDS
  auto bad = [](const Mat& M) { for (double x : M.a) if (!std::isfinite(x)) return true; return false; };
  if (bad(A) || bad(B)) throw Error(ERR_INTERNAL, "truncate: non-finite input");
  if (bad(out.A) || bad(out.B)) { FILE* f = fopen("/tmp/orc_bad_B.txt", "w"); for (i64 i = 0; i < B.m; ++i) { for (i64 j = 0; j < B.n; ++j) fprintf(f, "%.17g ", B(i, j)); fprintf(f, "\n"); } fclose(f); }
  if (bad(out.A) || bad(out.B)) throw Error(ERR_INTERNAL, "truncate: non-finite output m=" + std::to_string(m) + " n=" + std::to_string(n) + " l=" + std::to_string(A.n) + " k=" + std::to_string(k) + " s0=" + std::to_string(s.empty()?0:s[0]) + " bad QB " + std::to_string(bad(QB)) + " RB " + std::to_string(bad(RB)) + " U " + std::to_string(bad(U)) + " Vh " + std::to_string(bad(Vh)));
#endif
  return out;
}

// Fig. rkadd: R2 <- trunc(R2 + alpha R1) with R1 = A B^T, R2 = C D^T:
// QR of [B D], Ahat = [alpha A, C] R_B^T, SVD, choose k, C = U(:,1:k),
// D = Q_B Vhat Sigma~^T.
static void rkadd(double alpha, const LowRank& R1, LowRank& R2, const TruncOpts& o) {
  if (R1.k() == 0) return;  // adding the zero matrix
  g_stats.rkadds++;
  Mat aA = R1.A;
  for (double& x : aA.a) x *= alpha;
  Mat As = hcat(aA, R2.A);
  Mat Bs = hcat(R1.B, R2.B);
  R2 = truncate(As, Bs, o);
}

// Fig. rowmerge: merge R_j = A_j B_j^T (common row cluster, consecutive
// column clusters) into one low-rank matrix.
static LowRank rowmerge(const std::vector<LowRank>& parts, const TruncOpts& o) {
  CatScope cat(1);
  i64 rows = parts[0].A.m;
  std::vector<Mat> Qs(parts.size());
  std::vector<i64> coff(parts.size() + 1, 0), roff(parts.size() + 1, 0);
  Mat Ahat(rows, 0);
  for (size_t j = 0; j < parts.size(); ++j) {
    Mat Rj;
    householder_qr(parts[j].B, Qs[j], Rj);   // B_j = Q_j R_j
    Mat AR = matmul(false, true, parts[j].A, Rj);
    Ahat = hcat(Ahat, AR);
    coff[j + 1] = coff[j] + Qs[j].n;
    roff[j + 1] = roff[j] + parts[j].B.m;
  }
  LowRank out;
  i64 cols = roff[parts.size()];
  g_stats.truncations++;
  g_stats.rowmerges++;
  if (Ahat.n == 0) {
    out.A = Mat(rows, 0);
    out.B = Mat(cols, 0);
    return out;
  }
  Mat U, Vh;
  std::vector<double> s;
  svd_thin(Ahat, U, s, Vh);
  i64 k = choose_rank(s, o.eps, o.max_rank);
  trace_trunc(rows, cols, -Ahat.n, k);
  out.A = Mat(rows, k);
  for (i64 j = 0; j < k; ++j)
    for (i64 i = 0; i < rows; ++i) out.A(i, j) = U(i, j);
  out.B = Mat(cols, k);
  for (size_t p = 0; p < parts.size(); ++p) {
    // block p of blockdiag(Q_j) Vhat Sigma~^T
    Mat VS(Qs[p].n, k);
    for (i64 j = 0; j < k; ++j)
      for (i64 i = 0; i < Qs[p].n; ++i) VS(i, j) = Vh(coff[p] + i, j) * s[(size_t)j];
    Mat blk = matmul(false, false, Qs[p], VS);
    set_rows(out.B, roff[p], blk);
  }
  return out;
}

// Fig. rkmerge: merge a p x q grid of low-rank blocks, block columns first
// (rowmerge of the adjoints), then the block row of merged columns.
static LowRank rkmerge(const std::vector<std::vector<LowRank>>& grid, const TruncOpts& o) {
  size_t p = grid.size(), q = grid[0].size();
  std::vector<LowRank> cols(q);
  for (size_t j = 0; j < q; ++j) {
    std::vector<LowRank> adj(p);
    for (size_t i = 0; i < p; ++i) {
      adj[i].A = grid[i][j].B;  // (R_ij)^* = B_ij A_ij^T
      adj[i].B = grid[i][j].A;
    }
    LowRank cj_adj = rowmerge(adj, o);  // (column j)^* = A' B'^T
    cols[j].A = cj_adj.B;               // column j = B' A'^T
    cols[j].B = cj_adj.A;
  }
  return rowmerge(cols, o);
}

// ---------------------------------------------------------------------------
// Cluster tree (Section 2, Definition "Cluster tree") by geometric bisection.
// ---------------------------------------------------------------------------
struct CNode {
  i64 off = 0, size = 0;
  int level = 0;
  int parent = -1;
  std::vector<int> sons;
  double bmin[3] = {0, 0, 0}, bmax[3] = {0, 0, 0};
};

struct CTree {
  int d = 0;
  std::vector<CNode> nodes;  // pre-order, root 0
  std::vector<i64> perm;     // perm[i] = original index of permuted index i
};

static int ctree_rec(CTree& T, const double* x, std::vector<i64>& idx, int level, int parent,
                     i64 leaf) {
  int id = (int)T.nodes.size();
  T.nodes.push_back(CNode());
  CNode nd;
  nd.level = level;
  nd.parent = parent;
  nd.size = (i64)idx.size();
  nd.off = (i64)T.perm.size();
  for (int a = 0; a < T.d; ++a) {
    nd.bmin[a] = INFINITY;
    nd.bmax[a] = -INFINITY;
  }
  for (i64 p : idx)
    for (int a = 0; a < T.d; ++a) {
      double v = x[p * T.d + a];
      nd.bmin[a] = std::min(nd.bmin[a], v);
      nd.bmax[a] = std::max(nd.bmax[a], v);
    }
  if ((i64)idx.size() <= leaf) {
    for (i64 p : idx) T.perm.push_back(p);
    T.nodes[(size_t)id] = nd;
    return id;
  }
  int dim = 0;
  double ext = nd.bmax[0] - nd.bmin[0];
  for (int a = 1; a < T.d; ++a) {
    double e = nd.bmax[a] - nd.bmin[a];
    if (e > ext) {
      ext = e;
      dim = a;
    }
  }
  double mid = (nd.bmin[dim] + nd.bmax[dim]) / 2.0;
  std::vector<i64> lo, hi;
  for (i64 p : idx) (x[p * T.d + dim] < mid ? lo : hi).push_back(p);
  if (lo.empty() || hi.empty()) throw Error(ERR_ARG, "cluster tree: cannot bisect (duplicate points)");
  T.nodes[(size_t)id] = nd;
  int s1 = ctree_rec(T, x, lo, level + 1, id, leaf);
  int s2 = ctree_rec(T, x, hi, level + 1, id, leaf);
  T.nodes[(size_t)id].sons = {s1, s2};
  return id;
}

static CTree* ctree_build(const double* coords, i64 n, int d, i64 leaf) {
  if (n <= 0 || d < 1 || d > 3 || leaf < 1) throw Error(ERR_ARG, "cluster tree: bad arguments");
  CTree* T = new CTree();
  T->d = d;
  std::vector<i64> idx((size_t)n);
  for (i64 i = 0; i < n; ++i) idx[(size_t)i] = i;
  ctree_rec(*T, coords, idx, 0, -1, leaf);
  return T;
}

// ---------------------------------------------------------------------------
// Block tree (Section 2, Definition "Block tree") with admissibility
// max(diam t, diam s) <= eta dist(t, s), dist > 0.
// ---------------------------------------------------------------------------
enum Kind { NONLEAF = 0, DENSE = 1, LOWRANK = 2 };

struct BNode {
  int t, s;
  int level;
  int parent;
  int kind;
  std::vector<int> sons;  // ordered (t'_i, s'_j), i major
};

struct BTree {
  const CTree* R;
  const CTree* C;
  std::vector<BNode> nodes;  // pre-order, root 0
};

static double diam(const CNode& c, int d) {
  double x = 0.0;
  for (int a = 0; a < d; ++a) {
    double e = c.bmax[a] - c.bmin[a];
    x += e * e;
  }
  return std::sqrt(x);
}

static double dist(const CNode& a, const CNode& b, int d) {
  double x = 0.0;
  for (int k = 0; k < d; ++k) {
    double g = std::max(0.0, std::max(a.bmin[k] - b.bmax[k], b.bmin[k] - a.bmax[k]));
    x += g * g;
  }
  return std::sqrt(x);
}

static int btree_rec(BTree& B, int t, int s, int level, int parent, double eta) {
  int id = (int)B.nodes.size();
  BNode nd{t, s, level, parent, NONLEAF, {}};
  B.nodes.push_back(nd);
  const CNode& ct = B.R->nodes[(size_t)t];
  const CNode& cs = B.C->nodes[(size_t)s];
  int d = B.R->d;
  double dst = dist(ct, cs, d);
  if (dst > 0.0 && std::max(diam(ct, d), diam(cs, d)) <= eta * dst) {
    B.nodes[(size_t)id].kind = LOWRANK;
    return id;
  }
  if (ct.sons.empty() || cs.sons.empty()) {
    B.nodes[(size_t)id].kind = DENSE;
    return id;
  }
  std::vector<int> sons;
  for (int t2 : ct.sons)
    for (int s2 : cs.sons) sons.push_back(btree_rec(B, t2, s2, level + 1, id, eta));
  B.nodes[(size_t)id].sons = sons;
  return id;
}

static BTree* btree_build(const CTree* R, const CTree* C, double eta) {
  if (R->d != C->d) throw Error(ERR_ARG, "block tree: dimension mismatch");
  BTree* B = new BTree();
  B->R = R;
  B->C = C;
  btree_rec(*B, 0, 0, 0, -1, eta);
  return B;
}

// Son of block b with row cluster t2 and column cluster s2.
static int child(const BTree& B, int b, int t2, int s2) {
  for (int c : B.nodes[(size_t)b].sons)
    if (B.nodes[(size_t)c].t == t2 && B.nodes[(size_t)c].s == s2) return c;
  throw Error(ERR_INTERNAL, "block tree: son not found");
}

// ---------------------------------------------------------------------------
// H-matrix (Section 2, Definition "Hierarchical matrix"): low-rank A_b B_b^T on
// admissible leaves, dense N_b on inadmissible leaves.
// ---------------------------------------------------------------------------
struct HMat {
  const BTree* bt;
  std::vector<Mat> N;      // per block, dense leaves only
  std::vector<LowRank> R;  // per block, admissible leaves only
  i64 rows(int b) const { return bt->R->nodes[(size_t)bt->nodes[(size_t)b].t].size; }
  i64 cols(int b) const { return bt->C->nodes[(size_t)bt->nodes[(size_t)b].s].size; }
  int kind(int b) const { return bt->nodes[(size_t)b].kind; }
  const CNode& tc(int b) const { return bt->R->nodes[(size_t)bt->nodes[(size_t)b].t]; }
  const CNode& sc(int b) const { return bt->C->nodes[(size_t)bt->nodes[(size_t)b].s]; }
};

static HMat* hmat_zero(const BTree* bt) {
  HMat* H = new HMat();
  H->bt = bt;
  H->N.resize(bt->nodes.size());
  H->R.resize(bt->nodes.size());
  for (size_t b = 0; b < bt->nodes.size(); ++b) {
    if (bt->nodes[b].kind == DENSE) H->N[b] = Mat(H->rows((int)b), H->cols((int)b));
    if (bt->nodes[b].kind == LOWRANK) {
      H->R[b].A = Mat(H->rows((int)b), 0);
      H->R[b].B = Mat(H->cols((int)b), 0);
    }
  }
  return H;
}

// Copy of a sparse matrix (original ordering) into the H-matrix format on the
// permuted index set.  Admissible blocks must hold no entry (rank 0,
// Section 3 opening paragraph).
static HMat* hmat_from_csr(const BTree* bt, i64 n, const i64* rowptr, const i64* colidx,
                           const double* val) {
  const CTree& R = *bt->R;
  if ((i64)R.perm.size() != n || (i64)bt->C->perm.size() != n) throw Error(ERR_ARG, "csr: size mismatch");
  HMat* H = hmat_zero(bt);
  std::vector<i64> ipc((size_t)n);
  for (i64 i = 0; i < n; ++i) ipc[(size_t)bt->C->perm[(size_t)i]] = i;
  i64 placed = 0;
  for (size_t b = 0; b < bt->nodes.size(); ++b) {
    if (bt->nodes[b].kind != DENSE) continue;
    const CNode& t = H->tc((int)b);
    const CNode& s = H->sc((int)b);
    Mat& N = H->N[b];
    for (i64 i = 0; i < t.size; ++i) {
      i64 p = R.perm[(size_t)(t.off + i)];
      for (i64 e = rowptr[p]; e < rowptr[p + 1]; ++e) {
        i64 j = ipc[(size_t)colidx[e]];
        if (j >= s.off && j < s.off + s.size) {
          N(i, j - s.off) += val[e];
          ++placed;
        }
      }
    }
  }
  if (placed != rowptr[n]) {
    delete H;
    throw Error(ERR_ARG, "csr: entries inside admissible blocks (rank > 0) are not supported");
  }
  return H;
}

static void hmat_to_dense(const HMat& H, Mat& D, i64 r0, i64 c0) {
  for (size_t b = 0; b < H.bt->nodes.size(); ++b) {
    const CNode& t = H.tc((int)b);
    const CNode& s = H.sc((int)b);
    if (H.kind((int)b) == DENSE) {
      for (i64 j = 0; j < s.size; ++j)
        for (i64 i = 0; i < t.size; ++i) D(t.off - r0 + i, s.off - c0 + j) = H.N[b](i, j);
    } else if (H.kind((int)b) == LOWRANK) {
      const LowRank& L = H.R[b];
      for (i64 j = 0; j < s.size; ++j)
        for (i64 i = 0; i < t.size; ++i) {
          double x = 0.0;
          for (i64 l = 0; l < L.k(); ++l) x += L.A(i, l) * L.B(j, l);
          D(t.off - r0 + i, s.off - c0 + j) = x;
        }
    }
  }
}

// ---------------------------------------------------------------------------
// Fig. addeval: Y|t <- Y|t + alpha G|_{t x s} X|s.  X and Y hold the rows of
// index ranges starting at xbase / ybase.
// ---------------------------------------------------------------------------
static void addeval(const HMat& G, int b, double alpha, const Mat& X, i64 xbase, Mat& Y, i64 ybase) {
  const CNode& t = G.tc(b);
  const CNode& s = G.sc(b);
  int kind = G.kind(b);
  if (kind == DENSE) {
    Mat Xs = rows_of(X, s.off - xbase, s.size);
    gemm_acc(false, false, alpha, G.N[(size_t)b], Xs, Y, t.off - ybase);
  } else if (kind == LOWRANK) {
    const LowRank& L = G.R[(size_t)b];
    if (L.k() == 0) return;
    Mat Xs = rows_of(X, s.off - xbase, s.size);
    Mat Zh(L.k(), X.n);
    gemm_acc(true, false, alpha, L.B, Xs, Zh);        // Zhat = alpha B^T X
    gemm_acc(false, false, 1.0, L.A, Zh, Y, t.off - ybase);  // Y += A Zhat
  } else {
    for (int c : G.bt->nodes[(size_t)b].sons) addeval(G, c, alpha, X, xbase, Y, ybase);
  }
}

// Fig. addevaltrans: X|s <- X|s + alpha G|_{t x s}^T Y|t.
static void addevaltrans(const HMat& G, int b, double alpha, const Mat& Y, i64 ybase, Mat& X, i64 xbase) {
  const CNode& t = G.tc(b);
  const CNode& s = G.sc(b);
  int kind = G.kind(b);
  if (kind == DENSE) {
    Mat Yt = rows_of(Y, t.off - ybase, t.size);
    gemm_acc(true, false, alpha, G.N[(size_t)b], Yt, X, s.off - xbase);
  } else if (kind == LOWRANK) {
    const LowRank& L = G.R[(size_t)b];
    if (L.k() == 0) return;
    Mat Yt = rows_of(Y, t.off - ybase, t.size);
    Mat Zh(L.k(), Y.n);
    gemm_acc(true, false, alpha, L.A, Yt, Zh);        // Zhat = alpha A^T Y
    gemm_acc(false, false, 1.0, L.B, Zh, X, s.off - xbase);  // X += B Zhat
  } else {
    for (int c : G.bt->nodes[(size_t)b].sons) addevaltrans(G, c, alpha, Y, ybase, X, xbase);
  }
}

// ---------------------------------------------------------------------------
// Targets of updates: a block of an H-matrix, or a temporary leaf matrix
// created by Fig. flush when (t, r) is a leaf but products are still pending.
// ---------------------------------------------------------------------------
struct Temp {
  int t, r;          // cluster ids (row tree, column tree)
  bool dense;
  Mat N;
  LowRank R;
};

struct Target {
  HMat* M = nullptr;  // block b of M, or
  int b = -1;
  Temp* tmp = nullptr;  // a temporary leaf
  const CTree* RT = nullptr;
  const CTree* CT = nullptr;
  int t() const { return tmp ? tmp->t : M->bt->nodes[(size_t)b].t; }
  int r() const { return tmp ? tmp->r : M->bt->nodes[(size_t)b].s; }
  bool has_sons() const { return !tmp && M->kind(b) == NONLEAF; }
  bool is_dense() const { return tmp ? tmp->dense : M->kind(b) == DENSE; }
  Mat& N() { return tmp ? tmp->N : M->N[(size_t)b]; }
  LowRank& R() { return tmp ? tmp->R : M->R[(size_t)b]; }
};

static Target target_of(HMat* M, int b) {
  Target z;
  z.M = M;
  z.b = b;
  z.RT = M->bt->R;
  z.CT = M->bt->C;
  return z;
}

static LowRank restrict_lr(const LowRank& L, i64 r0, i64 rn, i64 c0, i64 cn) {
  LowRank out;
  out.A = rows_of(L.A, r0, rn);
  out.B = rows_of(L.B, c0, cn);
  return out;
}

// Fig. rkupdate: G|_{t x s} <- blocktrunc(G|_{t x s} + alpha A B^T).
static void rkupdate(double alpha, const LowRank& R, Target z, const TruncOpts& o) {
  if (R.k() == 0) return;
  if (z.is_dense()) {
    gemm_acc(false, true, alpha, R.A, R.B, z.N());
  } else if (!z.has_sons()) {
    rkadd(alpha, R, z.R(), o);
  } else {
    const CNode& t = z.RT->nodes[(size_t)z.t()];
    const CNode& r = z.CT->nodes[(size_t)z.r()];
    for (int c : z.M->bt->nodes[(size_t)z.b].sons) {
      const CNode& t2 = z.RT->nodes[(size_t)z.M->bt->nodes[(size_t)c].t];
      const CNode& r2 = z.CT->nodes[(size_t)z.M->bt->nodes[(size_t)c].s];
      LowRank Rs = restrict_lr(R, t2.off - t.off, t2.size, r2.off - r.off, r2.size);
      rkupdate(alpha, Rs, target_of(z.M, c), o);
    }
  }
}

// ---------------------------------------------------------------------------
// Section 4: accumulators (Rhat_{t,r}, P_{t,r}) and Fig. addproduct / split /
// flush.
// ---------------------------------------------------------------------------
struct Pending {
  double alpha;
  const HMat* X;
  int xb;  // (t, s) in X's block tree
  const HMat* Y;
  int yb;  // (s, r) in Y's block tree
};

// An accumulator (t, r) with t or r a leaf cluster holds Rhat in standard
// representation (the representation Section 2 gives small blocks): adding a
// product to it is an exact addition, and the one truncation happens when it
// is flushed into an admissible leaf.  Such a block can never hold a pending
// product (that needs (t,s) and (s,r) to have sons), so it is never split.
// Every other accumulator holds Rhat in factorised form and adds products by
// rkadd (Fig. addproduct).
struct Acc {
  int t, r;
  bool dense = false;
  LowRank R;  // factorised Rhat
  Mat D;      // Rhat in standard representation (dense accumulators)
  std::vector<Pending> P;
};

// The literal form of Section 4 (mode 2 of orc_hmul and orc_hlu): every
// accumulator holds Rhat factorised, whatever its clusters, and each leaf case
// of Fig. addproduct adds its product by rkadd, a truncation per product; the
// flush then applies Rhat by rkupdate.  It is kept beside the default reading
// (dense accumulators for blocks with a leaf cluster) so that the two can be
// compared: they represent the same sum and differ by the extra truncations.
static bool g_literal_acc = false;
struct LiteralAccScope {
  bool old;
  explicit LiteralAccScope(bool on) : old(g_literal_acc) { g_literal_acc = on; }
  ~LiteralAccScope() { g_literal_acc = old; }
};

static bool acc_is_dense(int t, int r, const CTree& RT, const CTree& CT) {
  if (g_literal_acc) return false;
  return RT.nodes[(size_t)t].sons.empty() || CT.nodes[(size_t)r].sons.empty();
}

static Acc acc_empty(int t, int r, const CTree& RT, const CTree& CT) {
  bool dense = acc_is_dense(t, r, RT, CT);
  Acc a;
  a.t = t;
  a.r = r;
  a.dense = dense;
  if (dense) {
    a.D = Mat(RT.nodes[(size_t)t].size, CT.nodes[(size_t)r].size);
  } else {
    a.R.A = Mat(RT.nodes[(size_t)t].size, 0);
    a.R.B = Mat(CT.nodes[(size_t)r].size, 0);
  }
  return a;
}

// Low-rank factors Ahat Bhat^T of X|_{t x s} Y|_{s x r} when (t,s) or (s,r)
// is a leaf: the four leaf cases of Fig. addproduct.  alpha is not applied.
static LowRank leaf_product(const HMat& X, int xb, const HMat& Y, int yb) {
  const CNode& t = X.tc(xb);
  const CNode& s = X.sc(xb);
  const CNode& r = Y.sc(yb);
  LowRank P;
  if (X.kind(xb) == DENSE) {
    const Mat& Nx = X.N[(size_t)xb];
    if (t.size <= s.size) {
      P.A = identity(t.size);
      P.B = Mat(r.size, t.size);
      Mat NxT = transpose(Nx);  // s x t
      addevaltrans(Y, yb, 1.0, NxT, s.off, P.B, r.off);
    } else {
      P.A = Nx;
      P.B = Mat(r.size, s.size);
      addevaltrans(Y, yb, 1.0, identity(s.size), s.off, P.B, r.off);
    }
  } else if (Y.kind(yb) == DENSE) {
    const Mat& Ny = Y.N[(size_t)yb];
    if (r.size <= s.size) {
      P.B = identity(r.size);
      P.A = Mat(t.size, r.size);
      addeval(X, xb, 1.0, Ny, s.off, P.A, t.off);
    } else {
      P.B = transpose(Ny);  // r x s
      P.A = Mat(t.size, s.size);
      addeval(X, xb, 1.0, identity(s.size), s.off, P.A, t.off);
    }
  } else if (X.kind(xb) == LOWRANK) {
    const LowRank& L = X.R[(size_t)xb];
    P.A = L.A;
    P.B = Mat(r.size, L.k());
    if (L.k() > 0) addevaltrans(Y, yb, 1.0, L.B, s.off, P.B, r.off);
  } else {
    const LowRank& L = Y.R[(size_t)yb];
    P.B = L.B;
    P.A = Mat(t.size, L.k());
    if (L.k() > 0) addeval(X, xb, 1.0, L.A, s.off, P.A, t.off);
  }
  return P;
}

static bool is_leaf(const HMat& H, int b) { return H.kind(b) != NONLEAF; }

// Fig. addproduct.
static void addproduct(double alpha, const HMat& X, int xb, const HMat& Y, int yb, Acc& acc,
                       const TruncOpts& o) {
  if (X.bt->nodes[(size_t)xb].s != Y.bt->nodes[(size_t)yb].t) throw Error(ERR_INTERNAL, "addproduct: s mismatch");
  if (is_leaf(X, xb) || is_leaf(Y, yb)) {
    g_stats.addproducts++;
    LowRank P = leaf_product(X, xb, Y, yb);
    if (acc.dense)
      gemm_acc(false, true, alpha, P.A, P.B, acc.D);
    else
      rkadd(alpha, P, acc.R, o);
  } else {
    g_stats.pending++;
    acc.P.push_back(Pending{alpha, &X, xb, &Y, yb});
  }
}

// Fig. split: accumulators for the sons (t', r') inherit Rhat|_{t' x r'};
// each pending product is expanded over s' in sons(s) by addproduct.
static std::vector<std::vector<Acc>> split(const Acc& acc, const CTree& RT, const CTree& CT,
                                           const TruncOpts& o) {
  if (acc.dense) throw Error(ERR_INTERNAL, "split: dense accumulator");
  const CNode& t = RT.nodes[(size_t)acc.t];
  const CNode& r = CT.nodes[(size_t)acc.r];
  std::vector<std::vector<Acc>> sons(t.sons.size());
  for (size_t i = 0; i < t.sons.size(); ++i) {
    for (size_t j = 0; j < r.sons.size(); ++j) {
      const CNode& t2 = RT.nodes[(size_t)t.sons[i]];
      const CNode& r2 = CT.nodes[(size_t)r.sons[j]];
      bool dense = acc_is_dense(t.sons[i], r.sons[j], RT, CT);
      Acc a;
      a.t = t.sons[i];
      a.r = r.sons[j];
      a.dense = dense;
      LowRank Rs = restrict_lr(acc.R, t2.off - t.off, t2.size, r2.off - r.off, r2.size);
      if (dense) {
        a.D = Mat(t2.size, r2.size);
        if (Rs.k() > 0) gemm_acc(false, true, 1.0, Rs.A, Rs.B, a.D);
      } else {
        a.R = std::move(Rs);
      }
      for (const Pending& p : acc.P) {
        const BNode& xn = p.X->bt->nodes[(size_t)p.xb];
        const CNode& s = p.X->bt->C->nodes[(size_t)xn.s];
        for (int s2 : s.sons) {
          int xb2 = child(*p.X->bt, p.xb, a.t, s2);
          int yb2 = child(*p.Y->bt, p.yb, s2, a.r);
          addproduct(p.alpha, *p.X, xb2, *p.Y, yb2, a, o);
        }
      }
      sons[i].push_back(std::move(a));
    }
  }
  return sons;
}

// Fig. flush: add everything held by the accumulator to Z.
static void flush(Acc& acc, Target z, const TruncOpts& o) {
  const CTree& RT = *z.RT;
  const CTree& CT = *z.CT;
  if (acc.dense) {
    // t or r is a leaf cluster, so (t, r) is a leaf of Z and nothing is
    // pending.  Dense leaf: exact addition.  Admissible leaf: one rkadd of the
    // accumulated matrix D, factorised as I D^T or D I^T (smaller side as rank).
    if (!acc.P.empty() || z.has_sons()) throw Error(ERR_INTERNAL, "flush: dense accumulator");
    if (z.is_dense()) {
      Mat& N = z.N();
      for (size_t i = 0; i < N.a.size(); ++i) N.a[i] += acc.D.a[i];
    } else {
      bool any = false;
      for (double x : acc.D.a) any = any || (x != 0.0);
      if (any) {
        LowRank F;
        if (acc.D.m <= acc.D.n) {
          F.A = identity(acc.D.m);
          F.B = transpose(acc.D);
        } else {
          F.A = acc.D;
          F.B = identity(acc.D.n);
        }
        rkadd(1.0, F, z.R(), o);
      }
    }
    for (double& x : acc.D.a) x = 0.0;
    return;
  }
  if (acc.P.empty()) {
    rkupdate(1.0, acc.R, z, o);
  } else if (z.has_sons()) {
    auto sons = split(acc, RT, CT, o);
    for (auto& row : sons)
      for (Acc& a : row) flush(a, target_of(z.M, child(*z.M->bt, z.b, a.t, a.r)), o);
  } else {
    // (t, r) is a leaf but products are pending: temporary son matrices.
    const CNode& t = RT.nodes[(size_t)acc.t];
    const CNode& r = CT.nodes[(size_t)acc.r];
    std::vector<std::vector<Temp>> tmp(t.sons.size());
    for (size_t i = 0; i < t.sons.size(); ++i)
      for (size_t j = 0; j < r.sons.size(); ++j) {
        const CNode& t2 = RT.nodes[(size_t)t.sons[i]];
        const CNode& r2 = CT.nodes[(size_t)r.sons[j]];
        Temp T;
        T.t = t.sons[i];
        T.r = r.sons[j];
        T.dense = z.is_dense();
        if (T.dense) {
          Mat& N = z.N();
          T.N = Mat(t2.size, r2.size);
          for (i64 c = 0; c < r2.size; ++c)
            for (i64 rr = 0; rr < t2.size; ++rr)
              T.N(rr, c) = N(t2.off - t.off + rr, r2.off - r.off + c);
        } else {
          T.R = restrict_lr(z.R(), t2.off - t.off, t2.size, r2.off - r.off, r2.size);
        }
        tmp[i].push_back(std::move(T));
      }
    auto sons = split(acc, RT, CT, o);
    for (size_t i = 0; i < sons.size(); ++i)
      for (size_t j = 0; j < sons[i].size(); ++j) {
        Target zt;
        zt.tmp = &tmp[i][j];
        zt.RT = &RT;
        zt.CT = &CT;
        flush(sons[i][j], zt, o);
      }
    if (z.is_dense()) {
      Mat& N = z.N();
      for (size_t i = 0; i < tmp.size(); ++i)
        for (size_t j = 0; j < tmp[i].size(); ++j) {
          const CNode& t2 = RT.nodes[(size_t)tmp[i][j].t];
          const CNode& r2 = CT.nodes[(size_t)tmp[i][j].r];
          for (i64 c = 0; c < r2.size; ++c)
            for (i64 rr = 0; rr < t2.size; ++rr)
              N(t2.off - t.off + rr, r2.off - r.off + c) = tmp[i][j].N(rr, c);
        }
    } else {
      std::vector<std::vector<LowRank>> grid(tmp.size());
      for (size_t i = 0; i < tmp.size(); ++i)
        for (size_t j = 0; j < tmp[i].size(); ++j) grid[i].push_back(tmp[i][j].R);
      z.R() = rkmerge(grid, o);
    }
  }
  acc.R.A = Mat(acc.R.A.m, 0);
  acc.R.B = Mat(acc.R.B.m, 0);
  acc.P.clear();
}

// ---------------------------------------------------------------------------
// Standard multiplication (Section 4 before "Accumulated updates"): each
// low-rank product is added at once by rkupdate; temporaries + rkmerge where
// Z is coarser than the product.
// ---------------------------------------------------------------------------
static void mult_std(double alpha, const HMat& X, int xb, const HMat& Y, int yb, Target z,
                     const TruncOpts& o) {
  if (is_leaf(X, xb) || is_leaf(Y, yb)) {
    g_stats.addproducts++;
    LowRank P = leaf_product(X, xb, Y, yb);
    rkupdate(alpha, P, z, o);
    return;
  }
  const CTree& RT = *z.RT;
  const CTree& CT = *z.CT;
  const CNode& s = X.sc(xb);
  if (z.has_sons()) {
    for (int c : z.M->bt->nodes[(size_t)z.b].sons) {
      int t2 = z.M->bt->nodes[(size_t)c].t, r2 = z.M->bt->nodes[(size_t)c].s;
      for (int s2 : s.sons)
        mult_std(alpha, X, child(*X.bt, xb, t2, s2), Y, child(*Y.bt, yb, s2, r2), target_of(z.M, c), o);
    }
    return;
  }
  const CNode& t = RT.nodes[(size_t)z.t()];
  const CNode& r = CT.nodes[(size_t)z.r()];
  std::vector<std::vector<Temp>> tmp(t.sons.size());
  for (size_t i = 0; i < t.sons.size(); ++i)
    for (size_t j = 0; j < r.sons.size(); ++j) {
      const CNode& t2 = RT.nodes[(size_t)t.sons[i]];
      const CNode& r2 = CT.nodes[(size_t)r.sons[j]];
      Temp T;
      T.t = t.sons[i];
      T.r = r.sons[j];
      T.dense = z.is_dense();
      if (T.dense) {
        T.N = Mat(t2.size, r2.size);
        for (i64 c = 0; c < r2.size; ++c)
          for (i64 rr = 0; rr < t2.size; ++rr) T.N(rr, c) = z.N()(t2.off - t.off + rr, r2.off - r.off + c);
      } else {
        T.R = restrict_lr(z.R(), t2.off - t.off, t2.size, r2.off - r.off, r2.size);
      }
      tmp[i].push_back(std::move(T));
    }
  for (size_t i = 0; i < tmp.size(); ++i)
    for (size_t j = 0; j < tmp[i].size(); ++j) {
      Target zt;
      zt.tmp = &tmp[i][j];
      zt.RT = &RT;
      zt.CT = &CT;
      for (int s2 : s.sons)
        mult_std(alpha, X, child(*X.bt, xb, tmp[i][j].t, s2), Y, child(*Y.bt, yb, s2, tmp[i][j].r), zt, o);
    }
  if (z.is_dense()) {
    for (size_t i = 0; i < tmp.size(); ++i)
      for (size_t j = 0; j < tmp[i].size(); ++j) {
        const CNode& t2 = RT.nodes[(size_t)tmp[i][j].t];
        const CNode& r2 = CT.nodes[(size_t)tmp[i][j].r];
        for (i64 c = 0; c < r2.size; ++c)
          for (i64 rr = 0; rr < t2.size; ++rr) z.N()(t2.off - t.off + rr, r2.off - r.off + c) = tmp[i][j].N(rr, c);
      }
  } else {
    std::vector<std::vector<LowRank>> grid(tmp.size());
    for (size_t i = 0; i < tmp.size(); ++i)
      for (size_t j = 0; j < tmp[i].size(); ++j) grid[i].push_back(tmp[i][j].R);
    z.R() = rkmerge(grid, o);
  }
}

// ---------------------------------------------------------------------------
// Dense leaf kernels: no-pivot LU, triangular solves with thin right-hand
// sides (the leaves of the H-solves below).
// ---------------------------------------------------------------------------
static void dense_lu(Mat& A) {
  CatScope cat(2);
  i64 n = A.m;
  g_stats.dense_lu++;
  count_flops(2.0 / 3.0 * (double)n * (double)n * (double)n);
  for (i64 k = 0; k < n; ++k) {
    double piv = A(k, k);
    if (piv == 0.0 || !std::isfinite(piv))
      throw Error(ERR_SINGULAR, "dense LU: zero or non-finite pivot " + std::to_string(piv) + " at row " +
                                    std::to_string(k) + " of " + std::to_string(n));
    for (i64 i = k + 1; i < n; ++i) A(i, k) /= piv;
    for (i64 j = k + 1; j < n; ++j) {
      double akj = A(k, j);
      if (akj == 0.0) continue;
      for (i64 i = k + 1; i < n; ++i) A(i, j) -= A(i, k) * akj;
    }
  }
}

// X(rows x0.., :) <- L^{-1} X with L the unit lower triangle of N.
static void dense_solve_L(const Mat& N, Mat& X, i64 x0) {
  CatScope cat(2);
  i64 n = N.m;
  count_flops((double)n * (double)n * (double)X.n);
  for (i64 c = 0; c < X.n; ++c)
    for (i64 k = 0; k < n; ++k) {
      double v = X(x0 + k, c);
      if (v == 0.0) continue;
      for (i64 i = k + 1; i < n; ++i) X(x0 + i, c) -= N(i, k) * v;
    }
}

// X <- U^{-1} X with U the upper triangle of N.
static void dense_solve_U(const Mat& N, Mat& X, i64 x0) {
  CatScope cat(2);
  i64 n = N.m;
  count_flops((double)n * (double)n * (double)X.n);
  for (i64 c = 0; c < X.n; ++c)
    for (i64 k = n - 1; k >= 0; --k) {
      double v = X(x0 + k, c) / N(k, k);
      X(x0 + k, c) = v;
      if (v == 0.0) continue;
      for (i64 i = 0; i < k; ++i) X(x0 + i, c) -= N(i, k) * v;
    }
}

// X <- U^{-T} X (U^T lower, non-unit).
static void dense_solve_Ut(const Mat& N, Mat& X, i64 x0) {
  CatScope cat(2);
  i64 n = N.m;
  count_flops((double)n * (double)n * (double)X.n);
  for (i64 c = 0; c < X.n; ++c)
    for (i64 k = 0; k < n; ++k) {
      double v = X(x0 + k, c);
      for (i64 i = 0; i < k; ++i) v -= N(i, k) * X(x0 + i, c);
      X(x0 + k, c) = v / N(k, k);
    }
}

// X <- L^{-T} X (L^T upper, unit).
static void dense_solve_Lt(const Mat& N, Mat& X, i64 x0) {
  CatScope cat(2);
  i64 n = N.m;
  count_flops((double)n * (double)n * (double)X.n);
  for (i64 c = 0; c < X.n; ++c)
    for (i64 k = n - 1; k >= 0; --k) {
      double v = X(x0 + k, c);
      for (i64 i = k + 1; i < n; ++i) v -= N(i, k) * X(x0 + i, c);
      X(x0 + k, c) = v;
    }
}

// H-matrix triangular solves with a thin dense right-hand side X whose rows
// are the index range starting at xbase.  d is a diagonal block (t, t).
// Forward substitution X <- L_tt^{-1} X (L unit lower).
static void hsolve_L(const HMat& G, int d, Mat& X, i64 xbase) {
  if (G.kind(d) == DENSE) {
    dense_solve_L(G.N[(size_t)d], X, G.tc(d).off - xbase);
    return;
  }
  const CNode& t = G.tc(d);
  for (size_t i = 0; i < t.sons.size(); ++i) {
    hsolve_L(G, child(*G.bt, d, t.sons[i], t.sons[i]), X, xbase);
    for (size_t j = i + 1; j < t.sons.size(); ++j)
      addeval(G, child(*G.bt, d, t.sons[j], t.sons[i]), -1.0, X, xbase, X, xbase);
  }
}

// Backward substitution X <- U_tt^{-1} X.
static void hsolve_U(const HMat& G, int d, Mat& X, i64 xbase) {
  if (G.kind(d) == DENSE) {
    dense_solve_U(G.N[(size_t)d], X, G.tc(d).off - xbase);
    return;
  }
  const CNode& t = G.tc(d);
  for (size_t ii = t.sons.size(); ii-- > 0;) {
    hsolve_U(G, child(*G.bt, d, t.sons[ii], t.sons[ii]), X, xbase);
    for (size_t j = 0; j < ii; ++j)
      addeval(G, child(*G.bt, d, t.sons[j], t.sons[ii]), -1.0, X, xbase, X, xbase);
  }
}

// X <- U_tt^{-T} X (forward, with U^T lower).
static void hsolve_Ut(const HMat& G, int d, Mat& X, i64 xbase) {
  if (G.kind(d) == DENSE) {
    dense_solve_Ut(G.N[(size_t)d], X, G.tc(d).off - xbase);
    return;
  }
  const CNode& t = G.tc(d);
  for (size_t i = 0; i < t.sons.size(); ++i) {
    hsolve_Ut(G, child(*G.bt, d, t.sons[i], t.sons[i]), X, xbase);
    for (size_t j = i + 1; j < t.sons.size(); ++j)
      addevaltrans(G, child(*G.bt, d, t.sons[i], t.sons[j]), -1.0, X, xbase, X, xbase);
  }
}

// X <- L_tt^{-T} X (backward, with L^T upper unit).
static void hsolve_Lt(const HMat& G, int d, Mat& X, i64 xbase) {
  if (G.kind(d) == DENSE) {
    dense_solve_Lt(G.N[(size_t)d], X, G.tc(d).off - xbase);
    return;
  }
  const CNode& t = G.tc(d);
  for (size_t ii = t.sons.size(); ii-- > 0;) {
    hsolve_Lt(G, child(*G.bt, d, t.sons[ii], t.sons[ii]), X, xbase);
    for (size_t j = 0; j < ii; ++j)
      addevaltrans(G, child(*G.bt, d, t.sons[ii], t.sons[j]), -1.0, X, xbase, X, xbase);
  }
}

// ---------------------------------------------------------------------------
// H-LU with accumulated updates (Section 6, by analogy with Fig. invert).
// ---------------------------------------------------------------------------
static void trsm_L_acc(HMat& G, int d, int b, const TruncOpts& o);
static void trsm_U_acc(HMat& G, int d, int b, const TruncOpts& o);

// Solve L_tt X = G|_{t x r} in place (block b = (t, r), d = (t, t)).
static void trsm_L_acc(HMat& G, int d, int b, const TruncOpts& o) {
  int kind = G.kind(b);
  if (kind == DENSE) {
    hsolve_L(G, d, G.N[(size_t)b], G.tc(b).off);
  } else if (kind == LOWRANK) {
    if (G.R[(size_t)b].k() > 0) hsolve_L(G, d, G.R[(size_t)b].A, G.tc(b).off);
  } else {
    const CTree& T = *G.bt->R;
    const CNode& t = G.tc(b);
    const CNode& r = G.sc(b);
    for (int rj : r.sons) {
      std::vector<Acc> acc;
      for (int ti : t.sons)
        acc.push_back(acc_empty(ti, rj, T, *G.bt->C));
      for (size_t i = 0; i < t.sons.size(); ++i) {
        int bi = child(*G.bt, b, t.sons[i], rj);
        flush(acc[i], target_of(&G, bi), o);
        trsm_L_acc(G, child(*G.bt, d, t.sons[i], t.sons[i]), bi, o);
        for (size_t l = i + 1; l < t.sons.size(); ++l)
          addproduct(-1.0, G, child(*G.bt, d, t.sons[l], t.sons[i]), G, bi, acc[l], o);
      }
    }
  }
}

// Solve X U_tt = G|_{r x t} in place (block b = (r, t), d = (t, t)).
static void trsm_U_acc(HMat& G, int d, int b, const TruncOpts& o) {
  int kind = G.kind(b);
  if (kind == DENSE) {
    Mat W = transpose(G.N[(size_t)b]);
    hsolve_Ut(G, d, W, G.sc(b).off);
    G.N[(size_t)b] = transpose(W);
  } else if (kind == LOWRANK) {
    if (G.R[(size_t)b].k() > 0) hsolve_Ut(G, d, G.R[(size_t)b].B, G.sc(b).off);
  } else {
    const CNode& r = G.tc(b);
    const CNode& t = G.sc(b);
    for (int rj : r.sons) {
      std::vector<Acc> acc;
      for (int ti : t.sons)
        acc.push_back(acc_empty(rj, ti, *G.bt->R, *G.bt->C));
      for (size_t i = 0; i < t.sons.size(); ++i) {
        int bi = child(*G.bt, b, rj, t.sons[i]);
        flush(acc[i], target_of(&G, bi), o);
        trsm_U_acc(G, child(*G.bt, d, t.sons[i], t.sons[i]), bi, o);
        for (size_t l = i + 1; l < t.sons.size(); ++l)
          addproduct(-1.0, G, bi, G, child(*G.bt, d, t.sons[i], t.sons[l]), acc[l], o);
      }
    }
  }
}

static void lu_acc(HMat& G, int b, Acc& acc, const TruncOpts& o) {
  if (G.kind(b) == DENSE) {
    flush(acc, target_of(&G, b), o);
    dense_lu(G.N[(size_t)b]);
    return;
  }
  if (G.kind(b) != NONLEAF) throw Error(ERR_ARG, "H-LU: admissible diagonal block");
  const CTree& T = *G.bt->R;
  const CNode& t = G.tc(b);
  auto sub = split(acc, T, *G.bt->C, o);
  acc.R.A = Mat(acc.R.A.m, 0);
  acc.R.B = Mat(acc.R.B.m, 0);
  acc.P.clear();
  size_t p = t.sons.size();
  for (size_t i = 0; i < p; ++i) {
    int di = child(*G.bt, b, t.sons[i], t.sons[i]);
    lu_acc(G, di, sub[i][i], o);
    for (size_t j = i + 1; j < p; ++j) {
      int bij = child(*G.bt, b, t.sons[i], t.sons[j]);
      flush(sub[i][j], target_of(&G, bij), o);
      trsm_L_acc(G, di, bij, o);
    }
    for (size_t j = i + 1; j < p; ++j) {
      int bji = child(*G.bt, b, t.sons[j], t.sons[i]);
      flush(sub[j][i], target_of(&G, bji), o);
      trsm_U_acc(G, di, bji, o);
    }
    for (size_t j = i + 1; j < p; ++j)
      for (size_t l = i + 1; l < p; ++l)
        addproduct(-1.0, G, child(*G.bt, b, t.sons[j], t.sons[i]), G,
                   child(*G.bt, b, t.sons[i], t.sons[l]), sub[j][l], o);
  }
}

// ---------------------------------------------------------------------------
// H-Cholesky with accumulated updates (Section 6: treated "in a similar way"
// as the inversion).  G symmetric positive definite; afterwards the lower
// blocks and the lower triangles of the diagonal leaves hold L (G = L L^T) and
// the upper ones hold L^T, so that the LU's right solve X <- X U^{-1} with
// U = L^T is X L^{-T}.
// ---------------------------------------------------------------------------
// Lower Cholesky factor of a dense SPD leaf in place, its transpose mirrored
// into the strictly upper triangle.
static void dense_chol(Mat& A) {
  CatScope cat(2);
  i64 n = A.m;
  g_stats.dense_lu++;
  count_flops((double)n * (double)n * (double)n / 3.0);
  for (i64 k = 0; k < n; ++k) {
    double d = A(k, k);
    for (i64 j = 0; j < k; ++j) d -= A(k, j) * A(k, j);
    if (!(d > 0.0) || !std::isfinite(d))
      throw Error(ERR_SINGULAR, "dense Cholesky: non-positive pivot " + std::to_string(d) + " at row " +
                                    std::to_string(k));
    double lkk = std::sqrt(d);
    A(k, k) = lkk;
    for (i64 i = k + 1; i < n; ++i) {
      double v = A(i, k);
      for (i64 j = 0; j < k; ++j) v -= A(i, j) * A(k, j);
      A(i, k) = v / lkk;
    }
  }
  for (i64 j = 1; j < n; ++j)
    for (i64 i = 0; i < j; ++i) A(i, j) = A(j, i);
}

// G's block dst (s x t) <- G's block src (t x s) transposed, leaf by leaf
// (the block tree of one cluster tree is symmetric).
static void transpose_block(HMat& G, int src, int dst) {
  int kind = G.kind(src);
  if (kind == DENSE) {
    G.N[(size_t)dst] = transpose(G.N[(size_t)src]);
  } else if (kind == LOWRANK) {
    G.R[(size_t)dst].A = G.R[(size_t)src].B;
    G.R[(size_t)dst].B = G.R[(size_t)src].A;
  } else {
    const CNode& t = G.tc(src);
    const CNode& s = G.sc(src);
    for (int ti : t.sons)
      for (int sj : s.sons) transpose_block(G, child(*G.bt, src, ti, sj), child(*G.bt, dst, sj, ti));
  }
}

// chol(t): the block Cholesky recursion on the binary cluster tree with the
// accumulator split as for the LU: chol(t1); flush the (2,1) updates and solve
// L21 = G21 L11^{-T}; mirror L21^T into the (1,2) block; addproduct the Schur
// update -L21 L21^T without flush; chol(t2) takes the accumulator.  The (1,2)
// accumulator is not used (its updates are the transposes of the (2,1) ones).
static void chol_acc(HMat& G, int b, Acc& acc, const TruncOpts& o) {
  if (G.kind(b) == DENSE) {
    flush(acc, target_of(&G, b), o);
    dense_chol(G.N[(size_t)b]);
    return;
  }
  if (G.kind(b) != NONLEAF) throw Error(ERR_ARG, "H-Cholesky: admissible diagonal block");
  const CTree& T = *G.bt->R;
  const CNode& t = G.tc(b);
  if (t.sons.size() != 2) throw Error(ERR_ARG, "H-Cholesky: the cluster tree must be binary");
  auto sub = split(acc, T, *G.bt->C, o);
  acc.R.A = Mat(acc.R.A.m, 0);
  acc.R.B = Mat(acc.R.B.m, 0);
  acc.P.clear();
  int t1 = t.sons[0], t2 = t.sons[1];
  int b11 = child(*G.bt, b, t1, t1), b12 = child(*G.bt, b, t1, t2);
  int b21 = child(*G.bt, b, t2, t1), b22 = child(*G.bt, b, t2, t2);
  chol_acc(G, b11, sub[0][0], o);
  flush(sub[1][0], target_of(&G, b21), o);
  trsm_U_acc(G, b11, b21, o);  // G21 L11^{-T}: U = L11^T sits in the upper part of block b11
  transpose_block(G, b21, b12);
  addproduct(-1.0, G, b21, G, b12, sub[1][1], o);
  chol_acc(G, b22, sub[1][1], o);
}

// ---------------------------------------------------------------------------
// H-matrix inversion with accumulated updates (Section 6, Fig. invert).
// ---------------------------------------------------------------------------
// Inverse of a dense diagonal leaf: no-pivot LU, then U^{-1} L^{-1} applied to
// the identity (the paper assumes every principal submatrix invertible).
static void dense_inverse(Mat& A) {
  Mat X = identity(A.m);
  dense_lu(A);
  dense_solve_L(A, X, 0);
  dense_solve_U(A, X, 0);
  A = X;
}

// Every leaf of the subtree of block b set to zero (dense leaves zero,
// admissible leaves rank 0).
static void zero_subtree(HMat& G, int b) {
  if (G.kind(b) == DENSE) {
    Mat& N = G.N[(size_t)b];
    std::fill(N.a.begin(), N.a.end(), 0.0);
  } else if (G.kind(b) == LOWRANK) {
    G.R[(size_t)b].A = Mat(G.rows(b), 0);
    G.R[(size_t)b].B = Mat(G.cols(b), 0);
  } else {
    for (int c : G.bt->nodes[(size_t)b].sons) zero_subtree(G, c);
  }
}

// Fig. invert: G|_{t x t} <- (G|_{t x t} + pending updates in acc)^{-1}, with
// H (same block tree) as the auxiliary storage of H_12 and H_21.  Readings:
// the cluster tree is binary; a flushed accumulator is not used again (each
// product gets a fresh one); the last product, H_12 H_21', is accumulated for
// the block t_1 x t_1 and flushed into G_11 (the figure's index t_2 there is
// read as t_1, the block that H_11' overwrites).
static void invert_acc(HMat& G, HMat& H, int b, Acc& acc, const TruncOpts& o) {
  if (G.kind(b) == DENSE) {
    flush(acc, target_of(&G, b), o);
    dense_inverse(G.N[(size_t)b]);
    return;
  }
  if (G.kind(b) != NONLEAF) throw Error(ERR_ARG, "H-inverse: admissible diagonal block");
  const CTree& T = *G.bt->R;
  const CTree& C = *G.bt->C;
  const CNode& t = G.tc(b);
  if (t.sons.size() != 2) throw Error(ERR_ARG, "H-inverse: the cluster tree must be binary");
  int t1 = t.sons[0], t2 = t.sons[1];
  auto sub = split(acc, T, C, o);
  acc.R.A = Mat(acc.R.A.m, 0);
  acc.R.B = Mat(acc.R.B.m, 0);
  acc.P.clear();
  int b11 = child(*G.bt, b, t1, t1), b12 = child(*G.bt, b, t1, t2);
  int b21 = child(*G.bt, b, t2, t1), b22 = child(*G.bt, b, t2, t2);
  // 1. G_11 <- G_11^{-1}
  invert_acc(G, H, b11, sub[0][0], o);
  // 2. H_12 = G_11^{-1} G_12, H_21 = G_21 G_11^{-1} (after the pending updates
  //    of G_12 and G_21 are flushed)
  flush(sub[0][1], target_of(&G, b12), o);
  flush(sub[1][0], target_of(&G, b21), o);
  zero_subtree(H, b12);
  zero_subtree(H, b21);
  {
    Acc a = acc_empty(t1, t2, T, C);
    addproduct(1.0, G, b11, G, b12, a, o);
    flush(a, target_of(&H, b12), o);
  }
  {
    Acc a = acc_empty(t2, t1, T, C);
    addproduct(1.0, G, b21, G, b11, a, o);
    flush(a, target_of(&H, b21), o);
  }
  // 3. S = G_22 - H_21 G_12, left in the accumulator (not flushed)
  addproduct(-1.0, H, b21, G, b12, sub[1][1], o);
  // 4. G_22 <- S^{-1}
  invert_acc(G, H, b22, sub[1][1], o);
  // 5. G_12 <- H_12' = -H_12 S^{-1}, G_21 <- H_21' = -S^{-1} H_21
  zero_subtree(G, b12);
  zero_subtree(G, b21);
  {
    Acc a = acc_empty(t1, t2, T, C);
    addproduct(-1.0, H, b12, G, b22, a, o);
    flush(a, target_of(&G, b12), o);
  }
  {
    Acc a = acc_empty(t2, t1, T, C);
    addproduct(-1.0, G, b22, H, b21, a, o);
    flush(a, target_of(&G, b21), o);
  }
  // 6. G_11 <- H_11' = G_11^{-1} - H_12 H_21'
  {
    Acc a = acc_empty(t1, t1, T, C);
    addproduct(-1.0, H, b12, G, b21, a, o);
    flush(a, target_of(&G, b11), o);
  }
}

// The same six steps with every product applied at once by the standard
// multiplication (Section 4 before "Accumulated updates"): the standard
// H-inversion the accumulated one is compared with.
static void invert_std(HMat& G, HMat& H, int b, const TruncOpts& o) {
  if (G.kind(b) == DENSE) {
    dense_inverse(G.N[(size_t)b]);
    return;
  }
  if (G.kind(b) != NONLEAF) throw Error(ERR_ARG, "H-inverse: admissible diagonal block");
  const CNode& t = G.tc(b);
  if (t.sons.size() != 2) throw Error(ERR_ARG, "H-inverse: the cluster tree must be binary");
  int t1 = t.sons[0], t2 = t.sons[1];
  int b11 = child(*G.bt, b, t1, t1), b12 = child(*G.bt, b, t1, t2);
  int b21 = child(*G.bt, b, t2, t1), b22 = child(*G.bt, b, t2, t2);
  invert_std(G, H, b11, o);
  zero_subtree(H, b12);
  zero_subtree(H, b21);
  mult_std(1.0, G, b11, G, b12, target_of(&H, b12), o);
  mult_std(1.0, G, b21, G, b11, target_of(&H, b21), o);
  mult_std(-1.0, H, b21, G, b12, target_of(&G, b22), o);
  invert_std(G, H, b22, o);
  zero_subtree(G, b12);
  zero_subtree(G, b21);
  mult_std(-1.0, H, b12, G, b22, target_of(&G, b12), o);
  mult_std(-1.0, G, b22, H, b21, target_of(&G, b21), o);
  mult_std(-1.0, H, b12, G, b21, target_of(&G, b11), o);
}

// ---------------------------------------------------------------------------
// Standard H-LU: same recursion, every product applied at once (Remark after
// the complexity theorem: rkadd in addproduct becomes rkupdate).
// ---------------------------------------------------------------------------
static void trsm_L_std(HMat& G, int d, int b, const TruncOpts& o) {
  int kind = G.kind(b);
  if (kind == DENSE) {
    hsolve_L(G, d, G.N[(size_t)b], G.tc(b).off);
  } else if (kind == LOWRANK) {
    if (G.R[(size_t)b].k() > 0) hsolve_L(G, d, G.R[(size_t)b].A, G.tc(b).off);
  } else {
    const CNode& t = G.tc(b);
    const CNode& r = G.sc(b);
    for (int rj : r.sons)
      for (size_t i = 0; i < t.sons.size(); ++i) {
        int bi = child(*G.bt, b, t.sons[i], rj);
        trsm_L_std(G, child(*G.bt, d, t.sons[i], t.sons[i]), bi, o);
        for (size_t l = i + 1; l < t.sons.size(); ++l)
          mult_std(-1.0, G, child(*G.bt, d, t.sons[l], t.sons[i]), G, bi,
                   target_of(&G, child(*G.bt, b, t.sons[l], rj)), o);
      }
  }
}

static void trsm_U_std(HMat& G, int d, int b, const TruncOpts& o) {
  int kind = G.kind(b);
  if (kind == DENSE) {
    Mat W = transpose(G.N[(size_t)b]);
    hsolve_Ut(G, d, W, G.sc(b).off);
    G.N[(size_t)b] = transpose(W);
  } else if (kind == LOWRANK) {
    if (G.R[(size_t)b].k() > 0) hsolve_Ut(G, d, G.R[(size_t)b].B, G.sc(b).off);
  } else {
    const CNode& r = G.tc(b);
    const CNode& t = G.sc(b);
    for (int rj : r.sons)
      for (size_t i = 0; i < t.sons.size(); ++i) {
        int bi = child(*G.bt, b, rj, t.sons[i]);
        trsm_U_std(G, child(*G.bt, d, t.sons[i], t.sons[i]), bi, o);
        for (size_t l = i + 1; l < t.sons.size(); ++l)
          mult_std(-1.0, G, bi, G, child(*G.bt, d, t.sons[i], t.sons[l]),
                   target_of(&G, child(*G.bt, b, rj, t.sons[l])), o);
      }
  }
}

static void lu_std(HMat& G, int b, const TruncOpts& o) {
  if (G.kind(b) == DENSE) {
    dense_lu(G.N[(size_t)b]);
    return;
  }
  if (G.kind(b) != NONLEAF) throw Error(ERR_ARG, "H-LU: admissible diagonal block");
  const CNode& t = G.tc(b);
  size_t p = t.sons.size();
  for (size_t i = 0; i < p; ++i) {
    int di = child(*G.bt, b, t.sons[i], t.sons[i]);
    lu_std(G, di, o);
    for (size_t j = i + 1; j < p; ++j) trsm_L_std(G, di, child(*G.bt, b, t.sons[i], t.sons[j]), o);
    for (size_t j = i + 1; j < p; ++j) trsm_U_std(G, di, child(*G.bt, b, t.sons[j], t.sons[i]), o);
    for (size_t j = i + 1; j < p; ++j)
      for (size_t l = i + 1; l < p; ++l)
        mult_std(-1.0, G, child(*G.bt, b, t.sons[j], t.sons[i]), G, child(*G.bt, b, t.sons[i], t.sons[l]),
                 target_of(&G, child(*G.bt, b, t.sons[j], t.sons[l])), o);
  }
}

// ---------------------------------------------------------------------------
// Preconditioner error ||I - (LU)^{-1} A||_2 (Section 7) by power iteration on
// E^T E with E = I - (LU)^{-1} A, on the permuted index set.
// ---------------------------------------------------------------------------
static void csr_perm_matvec(i64 n, const i64* rowptr, const i64* colidx, const double* val,
                            const std::vector<i64>& perm, const std::vector<i64>& iperm,
                            bool trans, const std::vector<double>& x, std::vector<double>& y) {
  y.assign((size_t)n, 0.0);
  for (i64 i = 0; i < n; ++i) {
    i64 p = perm[(size_t)i];
    for (i64 e = rowptr[p]; e < rowptr[p + 1]; ++e) {
      i64 j = iperm[(size_t)colidx[e]];
      if (!trans) y[(size_t)i] += val[e] * x[(size_t)j];
      else y[(size_t)j] += val[e] * x[(size_t)i];
    }
  }
}

}  // namespace orc

// ===========================================================================
// C interface (for ctypes)
// ===========================================================================
using namespace orc;

static thread_local std::string g_err;

template <class F>
static int guard(F f) {
  try {
    f();
    return OK;
  } catch (const Error& e) {
    g_err = e.what();
    return e.code;
  } catch (const std::exception& e) {
    g_err = e.what();
    return ERR_INTERNAL;
  }
}

struct orc_stats_t {
  int64_t truncations, rkadds, rowmerges, addproducts, pending, dense_lu;
  double flops, seconds, flops_trunc, flops_dense;
};

static void copy_stats(orc_stats_t* st) {
  if (!st) return;
  st->truncations = g_stats.truncations;
  st->rkadds = g_stats.rkadds;
  st->rowmerges = g_stats.rowmerges;
  st->addproducts = g_stats.addproducts;
  st->pending = g_stats.pending;
  st->dense_lu = g_stats.dense_lu;
  st->flops = g_stats.flops;
  st->seconds = g_stats.seconds;
  st->flops_trunc = g_stats.flops_trunc;
  st->flops_dense = g_stats.flops_dense;
}

static Mat from_colmajor(i64 m, i64 n, const double* a, i64 ld) {
  Mat M(m, n);
  for (i64 j = 0; j < n; ++j)
    for (i64 i = 0; i < m; ++i) M(i, j) = a[i + j * ld];
  return M;
}

static void to_colmajor(const Mat& M, double* a, i64 ld) {
  for (i64 j = 0; j < M.n; ++j)
    for (i64 i = 0; i < M.m; ++i) a[i + j * ld] = M(i, j);
}

extern "C" {

const char* orc_last_error() { return g_err.c_str(); }

void orc_stats_reset() { g_stats = Stats(); }
void orc_set_rank_rule(int rule) { g_rank_rule = rule == 1 ? 1 : 0; }
void orc_trace_enable(int on) {
  g_trace_on = on != 0;
  g_trace.clear();
}
int64_t orc_trace_size() { return (int64_t)g_trace.size() / 4; }
void orc_trace_get(int64_t* out) {
  for (size_t i = 0; i < g_trace.size(); ++i) out[i] = g_trace[i];
}
void orc_stats_get(orc_stats_t* st) { copy_stats(st); }

// Dense building blocks (exposed for pinning).
int orc_qr(int64_t m, int64_t n, const double* A, double* Q, double* R) {
  return guard([&] {
    Mat Qm, Rm;
    householder_qr(from_colmajor(m, n, A, m), Qm, Rm);
    to_colmajor(Qm, Q, m);
    to_colmajor(Rm, R, std::min(m, n));
  });
}

int orc_svd(int64_t m, int64_t n, const double* A, double* U, double* s, double* V) {
  return guard([&] {
    Mat Um, Vm;
    std::vector<double> sv;
    svd_thin(from_colmajor(m, n, A, m), Um, sv, Vm);
    to_colmajor(Um, U, m);
    to_colmajor(Vm, V, n);
    for (size_t i = 0; i < sv.size(); ++i) s[i] = sv[i];
  });
}

// Truncation of A B^T (A: m x l, B: n x l) -> C (m x k), D (n x k); C and D
// must hold min(m, n, l) columns.
int orc_trunc(int64_t m, int64_t n, int64_t l, const double* A, const double* B, double eps,
              int64_t max_rank, double* C, double* D, int64_t* k) {
  return guard([&] {
    TruncOpts o;
    o.eps = eps;
    o.max_rank = max_rank;
    LowRank R = truncate(from_colmajor(m, l, A, m), from_colmajor(n, l, B, n), o);
    *k = R.k();
    to_colmajor(R.A, C, m);
    to_colmajor(R.B, D, n);
  });
}

// Fig. rkadd on explicit factors: (C2, D2) <- trunc((C, D) + alpha (A, B)).
int orc_rkadd(int64_t m, int64_t n, double alpha, int64_t k1, const double* A, const double* B,
              int64_t k2, const double* C, const double* D, double eps, double* Cout,
              double* Dout, int64_t* kout) {
  return guard([&] {
    TruncOpts o;
    o.eps = eps;
    LowRank R1{from_colmajor(m, k1, A, m), from_colmajor(n, k1, B, n)};
    LowRank R2{from_colmajor(m, k2, C, m), from_colmajor(n, k2, D, n)};
    rkadd(alpha, R1, R2, o);
    *kout = R2.k();
    to_colmajor(R2.A, Cout, m);
    to_colmajor(R2.B, Dout, n);
  });
}

// Cluster tree.
int orc_ctree_build(const double* coords, int64_t n, int d, int64_t leaf, void** out) {
  return guard([&] { *out = ctree_build(coords, n, d, leaf); });
}
void orc_ctree_free(void* h) { delete (CTree*)h; }
int64_t orc_ctree_size(void* h) { return (int64_t)((CTree*)h)->nodes.size(); }
void orc_ctree_nodes(void* h, int64_t* off, int64_t* size, int* level, int* parent, int* nsons) {
  CTree* T = (CTree*)h;
  for (size_t i = 0; i < T->nodes.size(); ++i) {
    off[i] = T->nodes[i].off;
    size[i] = T->nodes[i].size;
    level[i] = T->nodes[i].level;
    parent[i] = T->nodes[i].parent;
    nsons[i] = (int)T->nodes[i].sons.size();
  }
}
void orc_ctree_perm(void* h, int64_t* perm) {
  CTree* T = (CTree*)h;
  for (size_t i = 0; i < T->perm.size(); ++i) perm[i] = T->perm[i];
}

// Block tree.
int orc_btree_build(void* rows, void* cols, double eta, void** out) {
  return guard([&] { *out = btree_build((CTree*)rows, (CTree*)cols, eta); });
}
void orc_btree_free(void* h) { delete (BTree*)h; }
int64_t orc_btree_size(void* h) { return (int64_t)((BTree*)h)->nodes.size(); }
void orc_btree_nodes(void* h, int* t, int* s, int* level, int* parent, int* kind) {
  BTree* B = (BTree*)h;
  for (size_t i = 0; i < B->nodes.size(); ++i) {
    t[i] = B->nodes[i].t;
    s[i] = B->nodes[i].s;
    level[i] = B->nodes[i].level;
    parent[i] = B->nodes[i].parent;
    kind[i] = B->nodes[i].kind;
  }
}

// H-matrices.
int orc_hmat_from_csr(void* bt, int64_t n, const int64_t* rowptr, const int64_t* colidx,
                      const double* val, void** out) {
  return guard([&] { *out = hmat_from_csr((BTree*)bt, n, rowptr, colidx, val); });
}
int orc_hmat_zero(void* bt, void** out) {
  return guard([&] { *out = hmat_zero((BTree*)bt); });
}
int orc_hmat_copy(void* h, void** out) {
  return guard([&] { *out = new HMat(*(HMat*)h); });
}
void orc_hmat_free(void* h) { delete (HMat*)h; }

// Leaf setters/getters (column-major).  For dense leaves data is rows x cols.
int orc_hmat_set_dense(void* h, int b, const double* data) {
  return guard([&] {
    HMat* H = (HMat*)h;
    if (H->kind(b) != DENSE) throw Error(ERR_ARG, "set_dense: not a dense leaf");
    H->N[(size_t)b] = from_colmajor(H->rows(b), H->cols(b), data, H->rows(b));
  });
}
int orc_hmat_set_lowrank(void* h, int b, int64_t k, const double* A, const double* B) {
  return guard([&] {
    HMat* H = (HMat*)h;
    if (H->kind(b) != LOWRANK) throw Error(ERR_ARG, "set_lowrank: not an admissible leaf");
    H->R[(size_t)b].A = from_colmajor(H->rows(b), k, A, H->rows(b));
    H->R[(size_t)b].B = from_colmajor(H->cols(b), k, B, H->cols(b));
  });
}
void orc_hmat_ranks(void* h, int64_t* ranks) {
  HMat* H = (HMat*)h;
  for (size_t b = 0; b < H->bt->nodes.size(); ++b)
    ranks[b] = H->kind((int)b) == LOWRANK ? H->R[b].k() : -1;
}
int orc_hmat_get_lowrank(void* h, int b, double* A, double* B) {
  return guard([&] {
    HMat* H = (HMat*)h;
    to_colmajor(H->R[(size_t)b].A, A, H->rows(b));
    to_colmajor(H->R[(size_t)b].B, B, H->cols(b));
  });
}
int orc_hmat_get_dense(void* h, int b, double* data) {
  return guard([&] {
    HMat* H = (HMat*)h;
    to_colmajor(H->N[(size_t)b], data, H->rows(b));
  });
}
int orc_hmat_to_dense(void* h, double* out) {
  return guard([&] {
    HMat* H = (HMat*)h;
    i64 m = H->bt->R->nodes[0].size, n = H->bt->C->nodes[0].size;
    Mat D(m, n);
    hmat_to_dense(*H, D, 0, 0);
    to_colmajor(D, out, m);
  });
}

// Y += alpha G X (trans = 0) or Y += alpha G^T X (trans = 1); X, Y column-major.
int orc_addeval(void* h, double alpha, int64_t ncol, const double* X, double* Y, int trans) {
  return guard([&] {
    HMat* H = (HMat*)h;
    i64 m = H->bt->R->nodes[0].size, n = H->bt->C->nodes[0].size;
    if (!trans) {
      Mat Xm = from_colmajor(n, ncol, X, n), Ym = from_colmajor(m, ncol, Y, m);
      addeval(*H, 0, alpha, Xm, 0, Ym, 0);
      to_colmajor(Ym, Y, m);
    } else {
      Mat Xm = from_colmajor(m, ncol, X, m), Ym = from_colmajor(n, ncol, Y, n);
      addevaltrans(*H, 0, alpha, Xm, 0, Ym, 0);
      to_colmajor(Ym, Y, n);
    }
  });
}

// Z <- blocktrunc(Z + alpha X Y).  mode 1 = accumulated (addproduct at the
// root, then flush), mode 2 = accumulated with the literal low-rank
// accumulators of Section 4, mode 0 = standard.
int orc_hmul(double alpha, void* X, void* Y, void* Z, double eps, int mode) {
  return guard([&] {
    TruncOpts o;
    o.eps = eps;
    HMat* Zm = (HMat*)Z;
    LiteralAccScope lit(mode == 2);
    auto t0 = std::chrono::steady_clock::now();
    if (mode >= 1) {
      Acc acc = acc_empty(0, 0, *Zm->bt->R, *Zm->bt->C);
      addproduct(alpha, *(HMat*)X, 0, *(HMat*)Y, 0, acc, o);
      flush(acc, target_of(Zm, 0), o);
    } else {
      mult_std(alpha, *(HMat*)X, 0, *(HMat*)Y, 0, target_of(Zm, 0), o);
    }
    g_stats.seconds += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  });
}

// In-place H-LU: unit lower L and upper U share the H-matrix.  mode 1 =
// accumulated, 2 = accumulated with the literal low-rank accumulators of
// Section 4, 0 = standard.
int orc_hlu(void* h, double eps, int mode) {
  return guard([&] {
    TruncOpts o;
    o.eps = eps;
    HMat* G = (HMat*)h;
    LiteralAccScope lit(mode == 2);
    auto t0 = std::chrono::steady_clock::now();
    if (mode >= 1) {
      Acc acc = acc_empty(0, 0, *G->bt->R, *G->bt->C);
      lu_acc(*G, 0, acc, o);
    } else {
      lu_std(*G, 0, o);
    }
    g_stats.seconds += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  });
}

// In-place H-Cholesky with accumulated updates (lower blocks: L, upper: L^T).
int orc_hchol(void* h, double eps) {
  return guard([&] {
    TruncOpts o;
    o.eps = eps;
    HMat* G = (HMat*)h;
    auto t0 = std::chrono::steady_clock::now();
    Acc acc = acc_empty(0, 0, *G->bt->R, *G->bt->C);
    chol_acc(*G, 0, acc, o);
    g_stats.seconds += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  });
}

// In-place H-inversion: accumulated (mode 1, Fig. invert) or standard (0).
int orc_hinv(void* h, double eps, int mode) {
  return guard([&] {
    TruncOpts o;
    o.eps = eps;
    HMat* G = (HMat*)h;
    std::unique_ptr<HMat> H(hmat_zero(G->bt));
    auto t0 = std::chrono::steady_clock::now();
    Acc acc = acc_empty(0, 0, *G->bt->R, *G->bt->C);
    if (mode == 1)
      invert_acc(*G, *H, 0, acc, o);
    else
      invert_std(*G, *H, 0, o);
    g_stats.seconds += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  });
}

// B <- (LU)^{-1} B (trans = 0) or (LU)^{-T} B (trans = 1), permuted order.
int orc_hsolve(void* h, int64_t nrhs, double* B, int trans) {
  return guard([&] {
    HMat* G = (HMat*)h;
    i64 n = G->bt->R->nodes[0].size;
    Mat X = from_colmajor(n, nrhs, B, n);
    if (!trans) {
      hsolve_L(*G, 0, X, 0);
      hsolve_U(*G, 0, X, 0);
    } else {
      hsolve_Ut(*G, 0, X, 0);
      hsolve_Lt(*G, 0, X, 0);
    }
    to_colmajor(X, B, n);
  });
}

// Preconditioned conjugate gradients (Hestenes and Stiefel 1952) for
// A x = b with the H-LU factors as the preconditioner, z = (LU)^{-1} r, for
// nrhs right-hand sides one after the other, in the permuted ordering.  B, X:
// n x nrhs column-major in the ORIGINAL ordering; x_0 = 0.  A column stops
// when ||r_k|| <= rtol ||b|| or after maxit steps; iters[c] and relres[c]
// (the true relative residual ||b - A x|| / ||b|| at the end) are returned.
// The preconditioned CG assumes a symmetric preconditioner: (LU)^{-1} of an
// SPD matrix is symmetric up to the truncation error of the factors.
int orc_pcg(void* h, int64_t n, const int64_t* rowptr, const int64_t* colidx, const double* val, int64_t nrhs,
            const double* B, double* X, double rtol, int64_t maxit, int64_t* iters, double* relres) {
  return guard([&] {
    HMat* G = (HMat*)h;
    const std::vector<i64>& perm = G->bt->R->perm;
    std::vector<i64> iperm((size_t)n);
    for (i64 i = 0; i < n; ++i) iperm[(size_t)perm[(size_t)i]] = i;
    auto dot = [&](const std::vector<double>& a, const std::vector<double>& b) {
      double t = 0.0;
      for (i64 i = 0; i < n; ++i) t += a[(size_t)i] * b[(size_t)i];
      return t;
    };
    auto precond = [&](const std::vector<double>& r, std::vector<double>& z) {
      Mat Z = from_colmajor(n, 1, r.data(), n);
      hsolve_L(*G, 0, Z, 0);
      hsolve_U(*G, 0, Z, 0);
      z.assign(Z.a.begin(), Z.a.end());
    };
    for (i64 c = 0; c < nrhs; ++c) {
      std::vector<double> b((size_t)n), x((size_t)n, 0.0), r, z, p, q;
      for (i64 i = 0; i < n; ++i) b[(size_t)i] = B[c * n + perm[(size_t)i]];
      r = b;
      double nb = std::sqrt(dot(b, b));
      precond(r, z);
      p = z;
      double rz = dot(r, z);
      i64 it = 0;
      while (it < maxit && std::sqrt(dot(r, r)) > rtol * nb) {
        csr_perm_matvec(n, rowptr, colidx, val, perm, iperm, false, p, q);
        double alpha = rz / dot(p, q);
        for (i64 i = 0; i < n; ++i) {
          x[(size_t)i] += alpha * p[(size_t)i];
          r[(size_t)i] -= alpha * q[(size_t)i];
        }
        precond(r, z);
        double rz1 = dot(r, z);
        double beta = rz1 / rz;
        rz = rz1;
        for (i64 i = 0; i < n; ++i) p[(size_t)i] = z[(size_t)i] + beta * p[(size_t)i];
        ++it;
      }
      csr_perm_matvec(n, rowptr, colidx, val, perm, iperm, false, x, q);
      double res = 0.0;
      for (i64 i = 0; i < n; ++i) res += (b[(size_t)i] - q[(size_t)i]) * (b[(size_t)i] - q[(size_t)i]);
      iters[c] = it;
      relres[c] = nb > 0.0 ? std::sqrt(res) / nb : 0.0;
      for (i64 i = 0; i < n; ++i) X[c * n + perm[(size_t)i]] = x[(size_t)i];
    }
  });
}

// ||I - (LU)^{-1} A||_2 by power iteration on E^T E; v0 is the (seeded) start
// vector in permuted order.  Stops after maxit steps or when the estimate
// changes by less than rtol relatively.
int orc_precond_error(void* h, int64_t n, const int64_t* rowptr, const int64_t* colidx,
                      const double* val, const double* v0, int maxit, double rtol,
                      double* err, int* iters) {
  return guard([&] {
    HMat* G = (HMat*)h;
    const std::vector<i64>& perm = G->bt->R->perm;
    std::vector<i64> iperm((size_t)n);
    for (i64 i = 0; i < n; ++i) iperm[(size_t)perm[(size_t)i]] = i;
    std::vector<double> v(v0, v0 + n), Av, w, z;
    auto normalize = [&](std::vector<double>& x) {
      double s = 0.0;
      for (double a : x) s += a * a;
      s = std::sqrt(s);
      if (s > 0) for (double& a : x) a /= s;
      return s;
    };
    normalize(v);
    double est = 0.0;
    int it = 0;
    for (; it < maxit; ++it) {
      // w = E v = v - (LU)^{-1} A v
      csr_perm_matvec(n, rowptr, colidx, val, perm, iperm, false, v, Av);
      Mat X = from_colmajor(n, 1, Av.data(), n);
      hsolve_L(*G, 0, X, 0);
      hsolve_U(*G, 0, X, 0);
      w.assign((size_t)n, 0.0);
      double nw = 0.0;
      for (i64 i = 0; i < n; ++i) {
        w[(size_t)i] = v[(size_t)i] - X(i, 0);
        nw += w[(size_t)i] * w[(size_t)i];
      }
      double new_est = std::sqrt(nw);
      // z = E^T w = w - A^T (LU)^{-T} w
      Mat Y = from_colmajor(n, 1, w.data(), n);
      hsolve_Ut(*G, 0, Y, 0);
      hsolve_Lt(*G, 0, Y, 0);
      std::vector<double> y(Y.a.begin(), Y.a.end());
      csr_perm_matvec(n, rowptr, colidx, val, perm, iperm, true, y, z);
      for (i64 i = 0; i < n; ++i) z[(size_t)i] = w[(size_t)i] - z[(size_t)i];
      bool done = it > 0 && std::fabs(new_est - est) <= rtol * new_est;
      est = new_est;
      if (normalize(z) == 0.0) {
        ++it;
        break;
      }
      v = z;
      if (done) {
        ++it;
        break;
      }
    }
    *err = est;
    *iters = it;
  });
}

}  // extern "C"
