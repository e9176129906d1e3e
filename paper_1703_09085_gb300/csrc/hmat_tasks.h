// hmat_tasks.h -- task descriptors shared by the host scheduler and the
// persistent device executor.
//
// The H-LU recursion (block LU with Schur complement, Section 6 of Boerm,
// arXiv:1703.09085, with the accumulators of Section 4) is unrolled on the host
// into a list of tasks in program order.  Each task is one small dense or
// low-rank operation executed by one CTA; its predecessors are the tasks that
// last wrote (or, for a write, last read) the memory objects it touches.
#pragma once
#include <stdint.h>

namespace hm {

enum TaskType : int32_t {
  T_NOP = 0,
  T_LU = 1,          // no-pivot LU of a dense leaf in place (a: N, m: size)
  T_TRSM = 2,        // thin right-hand side solve with a dense diagonal leaf (flags: which)
  T_HMV = 3,         // out += alpha op(G|subtree) in, over a leaf list (Fig. addeval / addevaltrans)
  T_DENSIFY = 4,     // out = op(G|subtree) as dense, over a leaf list
  T_GEMM = 5,        // C (+)= alpha A B^T  (widths from rank slots)
  T_ADD = 6,         // C += alpha op(A), dense m x n
  T_RKADD = 7,       // low-rank (c,d,rin) <- trunc((c,d) + alpha (a,b)), result in (e,f,rout)
  T_ROWMERGE = 8,    // Fig. rowmerge of two parts (a,b,wa) (c,d,wb) -> (e,f,rout)
  T_COPY = 9,        // copy m x n (ld) , optional transposition
  T_ZERO = 10,       // zero m x n (ld)
  T_RANKSET = 11,    // ranks[rout] = width (fixed or slot)
  T_INV = 12,        // inverse of a dense diagonal leaf in place (a: N, m: size, lda)
  T_CHOL = 13        // Cholesky of a dense SPD diagonal leaf in place, L^T mirrored above
};

// T_TRSM variants
enum TrsmKind : int32_t { TRSM_L = 0, TRSM_U = 1, TRSM_UT = 2, TRSM_LT = 3 };

// flags
enum TaskFlags : int32_t {
  F_TRANS = 1,        // T_HMV / T_DENSIFY: use G^T; T_ADD / T_COPY: transpose source
  F_ZERO_OUT = 2,     // T_HMV / T_GEMM: zero the output before accumulating
  F_A_IDENT = 4,      // T_RKADD: product factor A is the identity (width m)
  F_B_IDENT = 8,      // T_RKADD: product factor B is the identity (width n)
  F_B_TRANS = 16,     // T_RKADD: b points at B^T (w x n) instead of B (n x w)
  F_CHECK_ZERO = 32,  // T_RKADD: skip the truncation if the product is exactly zero
  F_SWAP_AB = 64      // T_ROWMERGE: parts are adjoints (the "A" role is the stored B)
};

// A width: >= 0 a fixed number of columns, < 0 the rank slot -(w+1).
static inline int32_t width_from_slot(int32_t slot) { return -(slot + 1); }

// Location of a matrix: offset in doubles into the H-matrix storage, or into
// the per-factorisation workspace arena when WS_BIT is set.  -1 = none.
static const int64_t WS_BIT = (int64_t)1 << 60;

struct HTask {
  int32_t type;
  int32_t flags;
  int32_t m, n;        // sizes (rows of A-side, rows of B-side / columns)
  int32_t p, q;        // extra sizes (T_TRSM: kind in p; T_ROWMERGE: rows of part 1 in p)
  int32_t wa, wb;      // widths of the product / parts
  int32_t rin, rout;   // rank slots read / written (-1: none)
  int32_t cap;         // column capacity of the output factors
  int32_t list_begin, list_len;  // leaf-list range (T_HMV / T_DENSIFY)
  int32_t lda, ldb, ldc, ldd, lde, ldf;
  int32_t pad0, pad1;
  double alpha;
  int64_t a, b, c, d, e, f;      // locations
  int64_t ws;                    // scratch location for this task (doubles)
};

// One leaf of a subtree for T_HMV / T_DENSIFY.
struct LeafRef {
  int32_t kind;        // 1 dense, 2 low rank
  int32_t rows, cols;  // #t', #s'
  int32_t roff, coff;  // offsets of t' in t and of s' in s
  int32_t rank_slot;   // low rank: rank slot
  int32_t lda, ldb;    // leading dimensions (dense: lda = rows)
  int64_t a, b;        // dense: N at a; low rank: U at a, V at b
};

// Gang tasks: a T_RKADD with pad1 = G > 1 is run by G CTAs together, the
// task list holding G consecutive copies (pad0 = the member's rank); only
// member 0 is a dependency of later tasks, and it finishes last.  q holds
// the stacked-width capacity L, list_begin the offset (doubles) of the gang
// region in the task's scratch.
#define HM_GANG_XCH 8  // doubles of exchange per member
#define HM_GANG_MIN_ROWS 128  // rows of a member's block
static inline int64_t gang_ws_doubles(int64_t m, int64_t n, int64_t L, int64_t G) {
  int64_t fl = 2 * G * L * L + 3 * (m + n) * L + G * (3 * G * L * L + L * L);
  return G * HM_GANG_XCH + (fl + 1) / 2 + G * 4 * L + G * 4 * L + 64;
}

// Device status word values (hmat_status numbering).
enum DevStatus : int32_t {
  DS_OK = 0, DS_SINGULAR = 3, DS_NONFINITE = 4, DS_RANK = 5, DS_TIMEOUT = 6, DS_INTERNAL = 9
};

}  // namespace hm
