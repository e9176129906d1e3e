// hmat_host.cpp -- host side of the GB300 H-matrix library and its C ABI.
//
// Trees are built on the host (they are integer work, negligible next to the
// arithmetic).  The numerical recursions -- H-LU with accumulated updates
// (Section 6 with Section 4's addproduct / split / flush), H-matrix
// multiplication (Section 4), the H-matrix solve and the H x thin-dense
// product (Fig. addeval) -- are unrolled by a symbolic
// pass into a task list in program order.  A task's predecessors are found by
// tracking, per memory object, its last writer and the readers since; scratch
// memory comes from size-classed free lists whose chunks are memory objects
// too, so reusing a chunk orders the new writer after the old readers.  The
// task list runs in one persistent kernel (hmat_kernels.cu).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <memory>
#include <stdexcept>
#include <string>
#include <thread>
#include <vector>

#include "hmat.h"
#include "hmat_kernels.h"
#include "hmat_tasks.h"

using namespace hm;

namespace {

struct HmError : std::runtime_error {
  int code;
  HmError(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define HM_CUDA(call)                                                                   \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      throw HmError(e_ == cudaErrorMemoryAllocation ? HMAT_ERR_NOMEM : HMAT_ERR_CUDA,   \
                    std::string(#call) + ": " + cudaGetErrorString(e_));                \
  } while (0)

thread_local std::string g_last_error;

template <class F>
hmat_status guarded(F f) {
  try {
    f();
    return HMAT_OK;
  } catch (const HmError& e) {
    g_last_error = e.what();
    return (hmat_status)e.code;
  } catch (const std::bad_alloc&) {
    g_last_error = "host allocation failed";
    return HMAT_ERR_NOMEM;
  } catch (const std::exception& e) {
    g_last_error = e.what();
    return HMAT_ERR_INTERNAL;
  }
}

void require(bool ok, const char* msg) {
  if (!ok) throw HmError(HMAT_ERR_ARG, msg);
}

const int64_t DEFAULT_MAX_RANK = 64;
const int64_t HM_LMAX_HOST = 256;  // largest stacked width a truncation task accepts
const int64_t TAG_SHIFT = 60;
inline int64_t tag_ws(int64_t off) { return off | ((int64_t)1 << TAG_SHIFT); }
inline int64_t tag_ext(int which, int64_t off) { return off | ((int64_t)(2 + which) << TAG_SHIFT); }

// Device buffer that frees itself.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DevBuf() {}
  explicit DevBuf(size_t b) { alloc(b); }
  void alloc(size_t b) {
    release();
    if (b == 0) b = 16;
    HM_CUDA(cudaMalloc(&p, b));
    bytes = b;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  ~DevBuf() { release(); }
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  template <class T>
  T* as() const {
    return (T*)p;
  }
};

template <class T>
void upload(DevBuf& b, const std::vector<T>& v, cudaStream_t st) {
  b.alloc(v.size() * sizeof(T));
  if (!v.empty()) HM_CUDA(cudaMemcpyAsync(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st));
}

}  // namespace

// ===========================================================================
// Context
// ===========================================================================
struct hmat_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int num_sms = 0;
  int blocks_per_sm = 1;
};

// ===========================================================================
// Trees (Section 2)
// ===========================================================================
struct CNodeH {
  int64_t off = 0, size = 0;
  int level = 0, parent = -1, nsons = 0;
  int son[2] = {-1, -1};
  double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
};

struct hmat_ctree {
  int d = 0;
  std::vector<CNodeH> nodes;
  std::vector<int64_t> perm;
};

struct BNodeH {
  int t = 0, s = 0, level = 0, parent = -1, kind = 0;
  int son0 = 0, nsons = 0;
};

struct hmat_btree {
  const hmat_ctree* R = nullptr;
  const hmat_ctree* C = nullptr;
  std::vector<BNodeH> nodes;
  std::vector<int> sons;
  int child(int b, int i, int j) const {
    const BNodeH& nd = nodes[(size_t)b];
    return sons[(size_t)(nd.son0 + i * C->nodes[(size_t)nd.s].nsons + j)];
  }
};

namespace {

// Geometric bisection on idx[lo, hi): tight box, longest side (first on
// ties), stable partition at the box midpoint.  idx ends as the permutation.
int ct_rec(hmat_ctree& T, const double* x, std::vector<int64_t>& idx, std::vector<int64_t>& tmp, int64_t lo,
           int64_t hi, int level, int parent, int64_t leaf) {
  int id = (int)T.nodes.size();
  T.nodes.emplace_back();
  CNodeH nd;
  nd.off = lo;
  nd.size = hi - lo;
  nd.level = level;
  nd.parent = parent;
  int d = T.d;
  for (int a = 0; a < d; ++a) {
    nd.lo[a] = INFINITY;
    nd.hi[a] = -INFINITY;
  }
  for (int64_t i = lo; i < hi; ++i)
    for (int a = 0; a < d; ++a) {
      double v = x[idx[(size_t)i] * d + a];
      nd.lo[a] = std::min(nd.lo[a], v);
      nd.hi[a] = std::max(nd.hi[a], v);
    }
  if (hi - lo > leaf) {
    int dim = 0;
    double ext = nd.hi[0] - nd.lo[0];
    for (int a = 1; a < d; ++a)
      if (nd.hi[a] - nd.lo[a] > ext) {
        ext = nd.hi[a] - nd.lo[a];
        dim = a;
      }
    double mid = (nd.lo[dim] + nd.hi[dim]) / 2.0;
    int64_t nlo = 0, nhi = 0;
    for (int64_t i = lo; i < hi; ++i)
      if (x[idx[(size_t)i] * d + dim] < mid) idx[(size_t)(lo + nlo++)] = idx[(size_t)i];
      else tmp[(size_t)(nhi++)] = idx[(size_t)i];
    for (int64_t i = 0; i < nhi; ++i) idx[(size_t)(lo + nlo + i)] = tmp[(size_t)i];
    if (nlo == 0 || nhi == 0) throw HmError(HMAT_ERR_ARG, "cluster tree: points cannot be bisected (duplicates?)");
    T.nodes[(size_t)id] = nd;
    int s0 = ct_rec(T, x, idx, tmp, lo, lo + nlo, level + 1, id, leaf);
    int s1 = ct_rec(T, x, idx, tmp, lo + nlo, hi, level + 1, id, leaf);
    T.nodes[(size_t)id].nsons = 2;
    T.nodes[(size_t)id].son[0] = s0;
    T.nodes[(size_t)id].son[1] = s1;
  } else {
    T.nodes[(size_t)id] = nd;
  }
  return id;
}

double box_diam(const CNodeH& c, int d) {
  double x = 0.0;
  for (int a = 0; a < d; ++a) {
    double e = c.hi[a] - c.lo[a];
    x += e * e;
  }
  return std::sqrt(x);
}

double box_dist(const CNodeH& p, const CNodeH& q, int d) {
  double x = 0.0;
  for (int a = 0; a < d; ++a) {
    double g = std::max(0.0, std::max(p.lo[a] - q.hi[a], q.lo[a] - p.hi[a]));
    x += g * g;
  }
  return std::sqrt(x);
}

int bt_rec(hmat_btree& B, int t, int s, int level, int parent, double eta) {
  int id = (int)B.nodes.size();
  BNodeH nd;
  nd.t = t;
  nd.s = s;
  nd.level = level;
  nd.parent = parent;
  B.nodes.push_back(nd);
  const CNodeH& ct = B.R->nodes[(size_t)t];
  const CNodeH& cs = B.C->nodes[(size_t)s];
  int d = B.R->d;
  double dst = box_dist(ct, cs, d);
  if (dst > 0.0 && std::max(box_diam(ct, d), box_diam(cs, d)) <= eta * dst) {
    B.nodes[(size_t)id].kind = 2;
    return id;
  }
  if (ct.nsons == 0 || cs.nsons == 0) {
    B.nodes[(size_t)id].kind = 1;
    return id;
  }
  std::vector<int> kids;
  for (int i = 0; i < ct.nsons; ++i)
    for (int j = 0; j < cs.nsons; ++j) kids.push_back(bt_rec(B, ct.son[i], cs.son[j], level + 1, id, eta));
  B.nodes[(size_t)id].son0 = (int)B.sons.size();
  B.nodes[(size_t)id].nsons = (int)kids.size();
  B.sons.insert(B.sons.end(), kids.begin(), kids.end());
  return id;
}

}  // namespace

// ===========================================================================
// H-matrix: device storage of every leaf
// ===========================================================================
struct SchedCache;

namespace hm_internal {
const void* mlp_weights(const hmat_mlp* M);
}

struct hmat {
  std::shared_ptr<SchedCache> cache;  // schedule kept by hmat_lu(reuse_schedule)
  std::vector<float> train;           // training pairs recorded by the last hmat_lu
  hmat_ctx* ctx = nullptr;
  int device = 0;                  // the context's device (the context may go first)
  const hmat_btree* bt = nullptr;
  int64_t n = 0;
  int64_t max_rank = DEFAULT_MAX_RANK;
  std::vector<int64_t> loc, vloc;  // per block: N or U offset, V offset (doubles)
  std::vector<int> cap, slot;
  std::vector<char> zero;          // statically known zero leaf
  int nslots = 0;
  DevBuf store;                    // leaves
  DevBuf ranks;                    // rank slots of the low-rank leaves
  int64_t store_doubles = 0;
  hmat_stats st{};
  int64_t rows(int b) const { return bt->R->nodes[(size_t)bt->nodes[(size_t)b].t].size; }
  int64_t cols(int b) const { return bt->C->nodes[(size_t)bt->nodes[(size_t)b].s].size; }
  int kind(int b) const { return bt->nodes[(size_t)b].kind; }
  const CNodeH& tc(int b) const { return bt->R->nodes[(size_t)bt->nodes[(size_t)b].t]; }
  const CNodeH& sc(int b) const { return bt->C->nodes[(size_t)bt->nodes[(size_t)b].s]; }
};

namespace {

// ===========================================================================
// Task scheduler
// ===========================================================================
// f(begin, end) over [0, n) split into contiguous chunks run by up to 8 host
// threads (one chunk, on the calling thread, for small n).  f must not throw.
template <class F>
void host_chunks(size_t n, F f) {
  unsigned nt = std::min(8u, std::max(1u, std::thread::hardware_concurrency()));
  if (n < ((size_t)1 << 16) || nt <= 1) {
    f((size_t)0, n);
    return;
  }
  size_t chunk = (n + nt - 1) / nt;
  std::vector<std::thread> th;
  for (unsigned t = 1; t < nt; ++t) {
    size_t b = t * chunk, e = std::min(n, b + chunk);
    if (b >= e) continue;
    try {
      th.emplace_back([&f, b, e] { f(b, e); });
    } catch (...) {  // no thread to be had: this chunk on the calling thread
      f(b, e);
    }
  }
  f((size_t)0, std::min(n, chunk));
  for (std::thread& x : th) x.join();
}

struct Sched {
  std::vector<HTask> tasks;
  std::vector<int64_t> dep_ptr{0};
  std::vector<int32_t> dep_idx;
  std::vector<LeafRef> leaves;
  struct Obj {
    int32_t writer = -1;
    std::vector<int32_t> readers;
  };
  std::vector<Obj> objs;
  int next_slot = 0;
  struct Chunk {
    int64_t off;
    int cls;
    int obj;
    int pool;
  };
  std::vector<Chunk> chunks;
  // Free lists per pool and size class.  Independent instances of a batch use
  // separate pools, so reusing scratch never orders one instance after another.
  std::vector<std::vector<std::deque<int>>> pools = std::vector<std::vector<std::deque<int>>>(1, std::vector<std::deque<int>>(64));
  int pool = 0;
  void set_pool(int p) {
    while ((int)pools.size() <= p) pools.emplace_back(64);
    pool = p;
  }
  int64_t ws_top = 0;
  std::vector<int32_t> depbuf;
  std::vector<float> feat;      // 4 static features per task (truncations only)
  std::vector<int32_t> level;   // longest chain of predecessors (ASAP level)
  std::vector<double> cpath;    // estimated flops of the longest chain ending here

  // Room for the tasks an H-LU of nblocks blocks emits (about 43 per block at
  // 64^3, three dependencies per task), so that the lists grow without being
  // copied; a larger schedule still grows as usual.
  void reserve_for_blocks(size_t nblocks) {
    size_t nt = 48 * nblocks;
    tasks.reserve(nt);
    dep_ptr.reserve(nt + 1);
    dep_idx.reserve(3 * nt);
    level.reserve(nt);
    cpath.reserve(nt);
    feat.reserve(4 * nt);
  }
  double est_total = 0.0;

  // Rough static cost of a task (ranks unknown on the host: a typical rank 8).
  double est_cost(const HTask& t) const {
    auto w = [](int x) { return x >= 0 ? (double)x : 8.0; };
    switch (t.type) {
      case T_LU: return 2.0 / 3.0 * t.m * (double)t.m * t.m;
      case T_TRSM: return (double)t.m * t.m * w(t.wa);
      case T_GEMM: return 2.0 * t.m * (double)t.n * w(t.wa);
      case T_ADD: case T_COPY: case T_ZERO: return (double)t.m * t.n;
      case T_HMV: {
        double f = 0.0;
        for (int i = 0; i < t.list_len; ++i) {
          const LeafRef& L = leaves[(size_t)(t.list_begin + i)];
          f += L.kind == 1 ? 2.0 * L.rows * L.cols * w(t.wa) : 16.0 * (L.rows + L.cols) * w(t.wa);
        }
        return f;
      }
      case T_DENSIFY: {
        double f = 0.0;
        for (int i = 0; i < t.list_len; ++i) f += (double)leaves[(size_t)(t.list_begin + i)].rows * leaves[(size_t)(t.list_begin + i)].cols;
        return f;
      }
      case T_RKADD: {
        double l = (t.flags & F_A_IDENT ? t.m : t.flags & F_B_IDENT ? t.n : w(t.wa)) + (t.rin >= 0 ? 8.0 : 0.0);
        return 4.0 * (t.m + t.n) * l * l + 30.0 * l * l * l;
      }
      case T_ROWMERGE: {
        double l = w(t.wa) + w(t.wb);
        return 4.0 * (t.m + t.p + t.q) * l * l + 30.0 * l * l * l;
      }
      default: return 0.0;
    }
  }

  int new_obj() {
    objs.emplace_back();
    return (int)objs.size() - 1;
  }
  int new_slot() { return next_slot++; }

  static int cls_of(int64_t dbl) {
    int c = 8;
    while (((int64_t)1 << c) < dbl) ++c;
    return c;
  }
  // Keep this many chunks of a class in flight before reusing one, so that
  // independent tasks rarely wait on each other through scratch reuse.
  static size_t keep(int c) {
    int64_t k = ((int64_t)1 << 25) >> c;
    return (size_t)std::max<int64_t>(4, std::min<int64_t>(512, k));
  }
  int alloc(int64_t dbl) {
    int c = cls_of(std::max<int64_t>(dbl, 1));
    auto& fl = pools[(size_t)pool][(size_t)c];
    if (fl.size() > keep(c)) {
      int id = fl.front();
      fl.pop_front();
      return id;
    }
    Chunk ch;
    ch.off = ws_top;
    ch.cls = c;
    ch.obj = new_obj();
    ch.pool = pool;
    ws_top += (int64_t)1 << c;
    chunks.push_back(ch);
    return (int)chunks.size() - 1;
  }
  void release(int id) { pools[(size_t)chunks[(size_t)id].pool][(size_t)chunks[(size_t)id].cls].push_back(id); }
  int64_t chunk_loc(int id) const { return tag_ws(chunks[(size_t)id].off); }
  int chunk_obj(int id) const { return chunks[(size_t)id].obj; }

  int32_t emit(const HTask& t, const std::vector<int>& reads, const std::vector<int>& writes) {
    int32_t id = (int32_t)tasks.size();
    depbuf.clear();
    for (int w : writes) {
      Obj& o = objs[(size_t)w];
      if (o.writer >= 0) depbuf.push_back(o.writer);
      depbuf.insert(depbuf.end(), o.readers.begin(), o.readers.end());
    }
    for (int r : reads) {
      Obj& o = objs[(size_t)r];
      if (o.writer >= 0) depbuf.push_back(o.writer);
    }
    std::sort(depbuf.begin(), depbuf.end());
    depbuf.erase(std::unique(depbuf.begin(), depbuf.end()), depbuf.end());
    dep_idx.insert(dep_idx.end(), depbuf.begin(), depbuf.end());
    dep_ptr.push_back((int64_t)dep_idx.size());
    int32_t lv = 0;
    double cp = 0.0;
    for (int32_t d : depbuf) {
      lv = std::max(lv, level[(size_t)d] + 1);
      cp = std::max(cp, cpath[(size_t)d]);
    }
    level.push_back(lv);
    double c = est_cost(t);
    cpath.push_back(cp + c);
    feat.insert(feat.end(), {0.f, 0.f, 0.f, 0.f});
    est_total += c;
    for (int r : reads) {
      Obj& o = objs[(size_t)r];
      if (o.readers.empty() || o.readers.back() != id) o.readers.push_back(id);
    }
    for (int w : writes) {
      Obj& o = objs[(size_t)w];
      o.writer = id;
      o.readers.clear();
    }
    tasks.push_back(t);
    return id;
  }

  // Members of a gang whose member 0 was just emitted as task id0, given
  // as tasks of their own (their leaf ranges differ): the same predecessors,
  // no object bookkeeping.
  void emit_gang_copies(int32_t id0, const HTask* members, int count) {
    for (int r = 0; r < count; ++r) {
      const HTask& t = members[r];
      int64_t d0 = dep_ptr[(size_t)id0], d1 = dep_ptr[(size_t)id0 + 1];
      for (int64_t k = d0; k < d1; ++k) dep_idx.push_back(dep_idx[(size_t)k]);
      dep_ptr.push_back((int64_t)dep_idx.size());
      level.push_back(level[(size_t)id0]);
      cpath.push_back(cpath[(size_t)id0]);
      for (int k = 0; k < 4; ++k) feat.push_back(feat[4 * (size_t)id0 + k]);
      tasks.push_back(t);
    }
  }

  // Members 1..G-1 of a gang whose member 0 was just emitted as task id0:
  // the same task with its rank, the same predecessors, and no object
  // bookkeeping (later tasks depend on member 0 alone, which finishes last).
  void emit_gang_members(int32_t id0, int G) {
    std::vector<HTask> m;
    for (int r = 1; r < G; ++r) {
      m.push_back(tasks[(size_t)id0]);
      m.back().pad0 = r;
    }
    emit_gang_copies(id0, m.data(), (int)m.size());
  }

  // Reorder the list by ASAP level (stable): still a topological order, and
  // tasks that can run together sit next to each other, so the in-order
  // dequeue of the executor sees the available parallelism.
  void order_by_level() {
    size_t n = tasks.size();
    // a counting sort by level, stable (tasks of one level keep their order)
    int32_t maxl = 0;
    for (size_t i = 0; i < n; ++i) maxl = std::max(maxl, level[i]);
    std::vector<int64_t> start((size_t)maxl + 2, 0);
    for (size_t i = 0; i < n; ++i) ++start[(size_t)level[i] + 1];
    for (size_t l = 1; l < start.size(); ++l) start[l] += start[l - 1];
    std::vector<int32_t> ord(n);
    for (size_t i = 0; i < n; ++i) ord[(size_t)start[(size_t)level[i]]++] = (int32_t)i;
    // the gathers below touch memory in random order: split over host threads
    std::vector<int32_t> pos(n);
    host_chunks(n, [&](size_t b, size_t e) {
      for (size_t i = b; i < e; ++i) pos[(size_t)ord[i]] = (int32_t)i;
    });
    std::vector<int64_t> p2(n + 1, 0);
    for (size_t i = 0; i < n; ++i) p2[i + 1] = p2[i] + (dep_ptr[(size_t)ord[i] + 1] - dep_ptr[(size_t)ord[i]]);
    std::vector<int32_t> d2((size_t)p2[n]);
    host_chunks(n, [&](size_t b, size_t e) {
      for (size_t i = b; i < e; ++i) {
        int64_t o = ord[i], at = p2[i];
        for (int64_t k = dep_ptr[(size_t)o]; k < dep_ptr[(size_t)o + 1]; ++k) d2[(size_t)at++] = pos[(size_t)dep_idx[(size_t)k]];
      }
    });
    dep_ptr.swap(p2);
    dep_idx.swap(d2);
    {
      // the tasks gathered into fresh storage (first touched by the threads that
      // fill it), then copied back in order
      std::unique_ptr<HTask[]> t2(new HTask[n]);
      host_chunks(n, [&](size_t b, size_t e) {
        for (size_t i = b; i < e; ++i) t2[i] = tasks[(size_t)ord[i]];
      });
      host_chunks(n, [&](size_t b, size_t e) { std::copy(t2.get() + b, t2.get() + e, tasks.begin() + (ptrdiff_t)b); });
    }
    std::vector<int32_t> l2(n);
    std::vector<double> c2(n);
    std::vector<float> f2(4 * n);
    host_chunks(n, [&](size_t b, size_t e) {
      for (size_t i = b; i < e; ++i) {
        l2[i] = level[(size_t)ord[i]];
        c2[i] = cpath[(size_t)ord[i]];
        for (int k = 0; k < 4; ++k) f2[4 * i + k] = feat[4 * (size_t)ord[i] + k];
      }
    });
    level.swap(l2);
    cpath.swap(c2);
    feat.swap(f2);
  }

  int32_t levels() const {
    int32_t m = 0;
    for (int32_t l : level) m = std::max(m, l + 1);
    return m;
  }
  double critical_flops() const {
    double m = 0.0;
    for (double c : cpath) m = std::max(m, c);
    return m;
  }
};

struct Hold {
  Sched* S;
  int chunk;
  Hold(Sched* s, int c) : S(s), chunk(c) {}
  ~Hold() { S->release(chunk); }
};
typedef std::shared_ptr<Hold> HoldP;

HTask blank(int type) {
  HTask t;
  std::memset(&t, 0, sizeof(t));
  t.type = type;
  t.rin = t.rout = -1;
  t.a = t.b = t.c = t.d = t.e = t.f = t.ws = -1;
  return t;
}

int64_t rk_ws(int64_t m, int64_t n, int64_t l) { return (2 * m + n) * l + 2 * l * l + 64; }

// Extra scratch of the randomised truncation (explicit M when it is the
// smaller form, sketch, Q, J, rotations, signs, Grams) -- the device layout of
// task_rkadd / trunc_rand.
const int64_t RMAX = 32;
int64_t rand_ws(int64_t m, int64_t n, int64_t l) {
  int64_t g = std::max(2 * l * l, l * RMAX);
  int64_t mx = (m * n <= (m + n) * l) ? m * n : 0;
  // FP32 path (m n <= 2^20): M, sketch, Q, J, QR of J as floats, then the
  // signs and the FP32 copies of the stacked factors
  int64_t f32 = (m * n <= ((int64_t)1 << 20)) ? (m * n + 2 * (m + n) * RMAX + n + (m + n) * l) / 2 + 64 : 0;
  // FP32 core: J and Q_J (n x RMAX floats each), W, Vrot, norms, permutation
  int64_t rot = (2 * n * RMAX + 4 * RMAX * RMAX + 2 * RMAX + 1) / 2;
  // FP32 factored path: SA, SB copies, Mhat, Q_B, panels, signs; then doubles
  int64_t fact = (2 * m * l + 2 * n * l + 2 * (m + l) * RMAX + l + 3) / 2 + 2 * l + l * RMAX + 16;
  return std::max(std::max(mx + 2 * m * RMAX + n * RMAX + RMAX * RMAX + (n + 1) / 2 + 1 + g + rot, f32), fact) + 64;
}

// ===========================================================================
// Symbolic arithmetic: the paper's procedures emitting tasks
// ===========================================================================

// Sizes of the small non-leaf blocks that accumulate densely when asked to:
// the smaller side at most DENSE_ACC_MIN (its identity-factor truncation then
// stays within the stacked-width limit with a full-capacity input rank), the
// larger at most DENSE_ACC_MAX.
const int64_t DENSE_ACC_MIN = 128;
const int64_t DENSE_ACC_MAX = 256;

// A low-rank matrix under construction: own storage, or a row-restricted view
// of another one (Section 3, "Splitting": no arithmetic).
struct SLow {
  int64_t u = -1, v = -1;
  int ldu = 0, ldv = 0;
  int wcode = 0;   // width: fixed (>= 0) or rank slot (< 0)
  int cap = 0;     // capacity of own storage (columns a result may have)
  int wmax = 0;    // largest width the current data can have (a view keeps its parent's)
  int obj = -1;
  bool own = false;
  bool zero = true;
  HoldP hold;
  int slot = -1;   // rank slot when own
};

struct SPend {
  double alpha;
  const hmat* X;
  int xb;
  const hmat* Y;
  int yb;
};

// Accumulator (Rhat_{t,r}, P_{t,r}) (Section 4).  Blocks with a leaf cluster
// on either side keep Rhat in standard representation (exact additions, one
// truncation when flushed into an admissible leaf); all others factorised,
// except, where the symbolic pass is told so, small blocks (dense_small):
// they too add their products exactly and truncate once per flush.  A dense
// accumulator split into its sons hands them views of its block (same
// storage, same dependency object).
struct SAcc {
  int t = 0, r = 0;
  bool dense = false;
  bool dzero = true;
  int64_t dloc = -1;
  int dld = 0;     // leading dimension of the dense block (a view keeps its parent's)
  int dobj = -1;
  HoldP dhold;
  SLow R;
  std::vector<SPend> P;
};

// Target of a flush: a block of an H-matrix, or a temporary low-rank matrix.
struct STarget {
  hmat* M = nullptr;
  int b = -1;
  SLow* tmp = nullptr;
  int t = 0, r = 0;
};

// Factors Ahat Bhat^T of a product in low-rank form.
struct SProd {
  bool zero = false;
  int wcode = 0, wcap = 0;
  int64_t a = -1, b = -1;
  int lda = 0, ldb = 0;
  bool aid = false, bid = false, btr = false;
  std::vector<int> objs;
  std::vector<HoldP> holds;
};

struct Sym {
  Sched& S;
  const hmat_ctree& RT;
  const hmat_ctree& CT;
  int64_t maxrank;
  bool mixed = false;
  bool dense_small = false;  // small non-leaf blocks also accumulate densely
  std::vector<const hmat*> mats;
  std::vector<int> objbase;
  std::vector<int64_t> hoffs;
  std::vector<int> slotbases;

  Sym(Sched& s, const hmat_ctree& rt, const hmat_ctree& ct, int64_t mr) : S(s), RT(rt), CT(ct), maxrank(mr) {}

  // A matrix whose storage sits hoff doubles from the run's storage base and
  // whose leaf rank slots start at slot slotbase (batches of instances).
  void add_matrix(const hmat* M, int64_t hoff = 0, int slotbase = 0) {
    mats.push_back(M);
    objbase.push_back((int)S.objs.size());
    hoffs.push_back(hoff);
    slotbases.push_back(slotbase);
    for (size_t b = 0; b < M->bt->nodes.size(); ++b) S.new_obj();
  }
  size_t mat_index(const hmat* M) const {
    for (size_t i = 0; i < mats.size(); ++i)
      if (mats[i] == M) return i;
    throw HmError(HMAT_ERR_INTERNAL, "unknown matrix");
  }
  int obj_of(const hmat* M, int b) const { return objbase[mat_index(M)] + b; }
  int64_t hl(const hmat* M, int b) const { return M->loc[(size_t)b] + hoffs[mat_index(M)]; }
  int64_t hv(const hmat* M, int b) const { return M->vloc[(size_t)b] + hoffs[mat_index(M)]; }
  int sl(const hmat* M, int b) const { return M->slot[(size_t)b] + slotbases[mat_index(M)]; }
  // Static features of the truncation just emitted for block (t, r) (the rank
  // predictor's first four inputs).
  void set_features(int t, int r) {
    const CNodeH& a = rc(t);
    const CNodeH& b = cc(r);
    int d = RT.d;
    // scale-free block descriptors: cluster sizes, diameter over distance
    // (bounded where the clusters touch), spatial dimension
    float* f = &S.feat[S.feat.size() - 4];
    double diam = 0.5 * (box_diam(a, d) + box_diam(b, d)) + 1e-300;
    f[0] = (float)(std::log2((double)std::max<int64_t>(a.size, 1)) / 10.0);
    f[1] = (float)(std::log2((double)std::max<int64_t>(b.size, 1)) / 10.0);
    f[2] = (float)(std::log(diam / (box_dist(a, b, d) + 1e-3 * diam)) / 4.0);
    f[3] = (float)d / 3.f;
  }
  const CNodeH& rc(int t) const { return RT.nodes[(size_t)t]; }
  const CNodeH& cc(int r) const { return CT.nodes[(size_t)r]; }
  int capof(int64_t m, int64_t n) const { return (int)std::min<int64_t>(std::min(m, n), maxrank); }

  // ---- leaves of a subtree --------------------------------------------------
  void collect(const hmat* M, int b, int64_t r0, int64_t c0, bool nonzero_only, std::vector<LeafRef>& out,
               std::vector<int>& objs) {
    const BNodeH& nd = M->bt->nodes[(size_t)b];
    if (nd.kind == 0) {
      for (int k = 0; k < nd.nsons; ++k)
        collect(M, M->bt->sons[(size_t)(nd.son0 + k)], r0, c0, nonzero_only, out, objs);
      return;
    }
    if (nonzero_only && M->zero[(size_t)b]) return;
    LeafRef L;
    std::memset(&L, 0, sizeof(L));
    L.kind = nd.kind;
    L.rows = (int)M->rows(b);
    L.cols = (int)M->cols(b);
    L.roff = (int)(M->tc(b).off - r0);
    L.coff = (int)(M->sc(b).off - c0);
    L.lda = (int)M->rows(b);
    L.ldb = (int)M->cols(b);
    L.a = hl(M, b);
    L.b = nd.kind == 2 ? hv(M, b) : -1;
    L.rank_slot = nd.kind == 2 ? sl(M, b) : -1;
    out.push_back(L);
    objs.push_back(obj_of(M, b));
  }

  // out (ldout) += alpha op(M|b) in (ldin), width wcode.  Returns false when
  // nothing was emitted (subtree statically zero and no zeroing requested).
  bool hmv(const hmat* M, int b, bool trans, double alpha, int64_t in, int ldin, int inobj, int64_t out, int ldout,
           int outobj, int wcode, bool zero_out, int out_rows) {
    std::vector<LeafRef> L;
    std::vector<int> reads;
    collect(M, b, M->tc(b).off, M->sc(b).off, true, L, reads);
    if (L.empty() && !zero_out) return false;
    HTask t = blank(T_HMV);
    t.flags = (trans ? F_TRANS : 0) | (zero_out ? F_ZERO_OUT : 0);
    t.m = out_rows;
    t.alpha = alpha;
    t.b = in;
    t.ldb = ldin;
    t.c = out;
    t.ldc = ldout;
    t.wa = wcode;
    if (inobj >= 0) reads.push_back(inobj);
    std::vector<int> cut = out_rows >= 4 * HM_GANG_MIN_ROWS ? hmv_cuts(L, trans, out_rows) : std::vector<int>();
    t.list_begin = (int)S.leaves.size();
    t.list_len = (int)L.size();
    S.leaves.insert(S.leaves.end(), L.begin(), L.end());
    if (cut.size() < 2) {
      S.emit(t, reads, {outobj});
      return true;
    }
    // a gang: member r takes the leaves [cut[r], cut[r+1]) and the output
    // rows [p, q) they write (no leaf crosses a member's rows)
    int G = (int)cut.size();
    std::vector<HTask> mem((size_t)G, t);
    for (int r = 0; r < G; ++r) {
      int b0 = cut[(size_t)r], b1 = r + 1 < G ? cut[(size_t)r + 1] : (int)L.size();
      HTask& m = mem[(size_t)r];
      m.pad0 = r;
      m.pad1 = G;
      m.list_begin = t.list_begin + b0;
      m.list_len = b1 - b0;
      m.p = r == 0 ? 0 : orow(L[(size_t)b0], trans);
      m.q = r + 1 < G ? orow(L[(size_t)b1], trans) : out_rows;
    }
    int32_t id0 = S.emit(mem[0], reads, {outobj});
    S.emit_gang_copies(id0, mem.data() + 1, G - 1);
    return true;
  }

  // Gang size of a rowmerge (m x (n0 + n1), stacked width at most l) of the
  // mixed form: large ones are truncated by a gang of CTAs like rkadd's.
  int merge_gang(int64_t m, int64_t n, int64_t l) const {
    if (!mixed || std::min(m, n) < 4 * HM_GANG_MIN_ROWS || l > 128) return 1;
    return (int)std::min<int64_t>(8, std::min(m, n) / HM_GANG_MIN_ROWS);
  }
  // Turn the rowmerge just emitted as task id0 into member 0 of a gang of G
  // (n = n0 + n1, q = the stacked-width capacity, the gang region at
  // base_ws in the task's scratch) and emit the other members.
  void make_merge_gang(int32_t id0, int G, int64_t l, int64_t base_ws) {
    HTask& g0 = S.tasks[(size_t)id0];
    g0.n = g0.p + g0.q;
    g0.q = (int)l;
    g0.pad0 = 0;
    g0.pad1 = G;
    g0.list_begin = (int32_t)base_ws;
    S.emit_gang_members(id0, G);
  }

  static int orow(const LeafRef& L, bool trans) { return trans ? L.coff : L.roff; }

  // Split points of an H x thin-dense product's leaf list for a gang: the
  // leaves sorted by their first output row, cut only where no earlier leaf
  // reaches past the next one's rows, the parts of about equal work.  Returns
  // the first leaf of every part (fewer than two: no gang).
  std::vector<int> hmv_cuts(std::vector<LeafRef>& L, bool trans, int out_rows) {
    std::vector<int> cut;
    if (L.size() < 8) return cut;
    std::vector<LeafRef> S(L);
    std::stable_sort(S.begin(), S.end(), [&](const LeafRef& a, const LeafRef& b) { return orow(a, trans) < orow(b, trans); });
    std::vector<double> work(S.size() + 1, 0.0);
    for (size_t i = 0; i < S.size(); ++i)
      work[i + 1] = work[i] + (S[i].kind == 1 ? (double)S[i].rows * S[i].cols : 16.0 * (S[i].rows + S[i].cols));
    int G = std::min(8, out_rows / HM_GANG_MIN_ROWS);
    cut.push_back(0);
    int reach = 0;  // largest end row of the leaves before i
    for (size_t i = 0; i < S.size() && (int)cut.size() < G; ++i) {
      int r0 = orow(S[i], trans);
      if (i > 0 && reach <= r0 && work[i] >= work.back() * (double)cut.size() / G) cut.push_back((int)i);
      reach = std::max(reach, r0 + (trans ? S[i].cols : S[i].rows));
    }
    if (cut.size() < 2) cut.clear();
    else L.swap(S);  // the gang's members take consecutive runs of the sorted list
    return cut;
  }

  bool subtree_zero(const hmat* M, int b) {
    const BNodeH& nd = M->bt->nodes[(size_t)b];
    if (nd.kind != 0) return M->zero[(size_t)b];
    for (int k = 0; k < nd.nsons; ++k)
      if (!subtree_zero(M, M->bt->sons[(size_t)(nd.son0 + k)])) return false;
    return true;
  }

  // ---- H-matrix solves with a thin right-hand side (rows of d's cluster) -----
  // kind: TRSM_L (L^{-1}), TRSM_U (U^{-1}), TRSM_UT (U^{-T}), TRSM_LT (L^{-T})
  void hsolve(const hmat* M, int d, int kind, int64_t x, int ldx, int xobj, int wcode) {
    const BNodeH& nd = M->bt->nodes[(size_t)d];
    if (nd.kind == 1) {
      HTask t = blank(T_TRSM);
      t.p = kind;
      t.m = (int)M->rows(d);
      t.a = hl(M, d);
      t.lda = (int)M->rows(d);
      t.b = x;
      t.ldb = ldx;
      t.wa = wcode;
      S.emit(t, {obj_of(M, d)}, {xobj});
      return;
    }
    if (nd.kind != 0) throw HmError(HMAT_ERR_ARG, "H-solve: admissible diagonal block");
    const CNodeH& t = rc(nd.t);
    int p = t.nsons;
    auto xoff = [&](int i) { return x + (rc(t.son[i]).off - t.off); };
    auto rows = [&](int i) { return (int)rc(t.son[i]).size; };
    if (kind == TRSM_L || kind == TRSM_UT) {
      for (int i = 0; i < p; ++i) {
        hsolve(M, M->bt->child(d, i, i), kind, xoff(i), ldx, xobj, wcode);
        for (int j = i + 1; j < p; ++j) {
          if (kind == TRSM_L)
            hmv(M, M->bt->child(d, j, i), false, -1.0, xoff(i), ldx, xobj, xoff(j), ldx, xobj, wcode, false, rows(j));
          else
            hmv(M, M->bt->child(d, i, j), true, -1.0, xoff(i), ldx, xobj, xoff(j), ldx, xobj, wcode, false, rows(j));
        }
      }
    } else {
      for (int i = p - 1; i >= 0; --i) {
        hsolve(M, M->bt->child(d, i, i), kind, xoff(i), ldx, xobj, wcode);
        for (int j = 0; j < i; ++j) {
          if (kind == TRSM_U)
            hmv(M, M->bt->child(d, j, i), false, -1.0, xoff(i), ldx, xobj, xoff(j), ldx, xobj, wcode, false, rows(j));
          else
            hmv(M, M->bt->child(d, i, j), true, -1.0, xoff(i), ldx, xobj, xoff(j), ldx, xobj, wcode, false, rows(j));
        }
      }
    }
  }

  // ---- products (Fig. addproduct, four leaf cases) -----------------------------
  int scratch(int64_t dbl, SProd& P) {
    int c = S.alloc(dbl);
    P.holds.push_back(std::make_shared<Hold>(&S, c));
    P.objs.push_back(S.chunk_obj(c));
    return c;
  }

  SProd leaf_product(const hmat* X, int xb, const hmat* Y, int yb) {
    SProd P;
    const CNodeH& t = X->tc(xb);
    const CNodeH& s = X->sc(xb);
    const CNodeH& r = Y->sc(yb);
    int nt = (int)t.size, ns = (int)s.size, nr = (int)r.size;
    int kx = X->kind(xb), ky = Y->kind(yb);
    if (kx == 1) {
      if (X->zero[(size_t)xb] || subtree_zero(Y, yb)) {
        P.zero = true;
        return P;
      }
      int xobj = obj_of(X, xb);
      if (nt <= ns) {
        // Ahat = I, Bhat = Y^T N_X^T (r x t)
        int cT = scratch((int64_t)ns * nt, P);
        HTask tc = blank(T_COPY);
        tc.flags = F_TRANS;
        tc.m = ns;
        tc.n = nt;
        tc.a = hl(X, xb);
        tc.lda = nt;
        tc.c = S.chunk_loc(cT);
        tc.ldc = ns;
        S.emit(tc, {xobj}, {S.chunk_obj(cT)});
        int cB = scratch((int64_t)nr * nt, P);
        hmv(Y, yb, true, 1.0, S.chunk_loc(cT), ns, S.chunk_obj(cT), S.chunk_loc(cB), nr, S.chunk_obj(cB), nt, true,
            nr);
        P.aid = true;
        P.b = S.chunk_loc(cB);
        P.ldb = nr;
        P.wcode = P.wcap = nt;
      } else {
        // Ahat = N_X (t x s), Bhat = Y^T (r x s)
        int cB = scratch((int64_t)nr * ns, P);
        densify(Y, yb, true, S.chunk_loc(cB), nr, S.chunk_obj(cB));
        P.a = hl(X, xb);
        P.lda = nt;
        P.objs.push_back(xobj);
        P.b = S.chunk_loc(cB);
        P.ldb = nr;
        P.wcode = P.wcap = ns;
      }
    } else if (ky == 1) {
      if (Y->zero[(size_t)yb] || subtree_zero(X, xb)) {
        P.zero = true;
        return P;
      }
      int yobj = obj_of(Y, yb);
      if (nr <= ns) {
        // Bhat = I, Ahat = X N_Y (t x r)
        int cA = scratch((int64_t)nt * nr, P);
        hmv(X, xb, false, 1.0, hl(Y, yb), ns, yobj, S.chunk_loc(cA), nt, S.chunk_obj(cA), nr, true, nt);
        P.bid = true;
        P.a = S.chunk_loc(cA);
        P.lda = nt;
        P.wcode = P.wcap = nr;
      } else {
        // Bhat = N_Y^T (given transposed), Ahat = X densified (t x s)
        int cA = scratch((int64_t)nt * ns, P);
        densify(X, xb, false, S.chunk_loc(cA), nt, S.chunk_obj(cA));
        P.a = S.chunk_loc(cA);
        P.lda = nt;
        P.b = hl(Y, yb);
        P.ldb = ns;
        P.btr = true;
        P.objs.push_back(yobj);
        P.wcode = P.wcap = ns;
      }
    } else if (kx == 2) {
      if (X->zero[(size_t)xb] || subtree_zero(Y, yb)) {
        P.zero = true;
        return P;
      }
      int xobj = obj_of(X, xb);
      int cx = X->cap[(size_t)xb];
      int wc = width_from_slot(sl(X, xb));
      int cB = scratch((int64_t)nr * cx, P);
      hmv(Y, yb, true, 1.0, hv(X, xb), ns, xobj, S.chunk_loc(cB), nr, S.chunk_obj(cB), wc, true, nr);
      P.a = hl(X, xb);
      P.lda = nt;
      P.objs.push_back(xobj);
      P.b = S.chunk_loc(cB);
      P.ldb = nr;
      P.wcode = wc;
      P.wcap = cx;
    } else {
      if (Y->zero[(size_t)yb] || subtree_zero(X, xb)) {
        P.zero = true;
        return P;
      }
      int yobj = obj_of(Y, yb);
      int cy = Y->cap[(size_t)yb];
      int wc = width_from_slot(sl(Y, yb));
      int cA = scratch((int64_t)nt * cy, P);
      hmv(X, xb, false, 1.0, hl(Y, yb), ns, yobj, S.chunk_loc(cA), nt, S.chunk_obj(cA), wc, true, nt);
      P.b = hv(Y, yb);
      P.ldb = nr;
      P.objs.push_back(yobj);
      P.a = S.chunk_loc(cA);
      P.lda = nt;
      P.wcode = wc;
      P.wcap = cy;
    }
    return P;
  }

  void densify(const hmat* M, int b, bool trans, int64_t out, int ldout, int outobj) {
    std::vector<LeafRef> L;
    std::vector<int> reads;
    collect(M, b, M->tc(b).off, M->sc(b).off, false, L, reads);
    HTask t = blank(T_DENSIFY);
    t.flags = trans ? F_TRANS : 0;
    t.c = out;
    t.ldc = ldout;
    t.list_begin = (int)S.leaves.size();
    t.list_len = (int)L.size();
    S.leaves.insert(S.leaves.end(), L.begin(), L.end());
    S.emit(t, reads, {outobj});
  }

  // ---- accumulators -------------------------------------------------------------
  SAcc acc_new(int t, int r) {
    SAcc a;
    a.t = t;
    a.r = r;
    int64_t m = rc(t).size, n = cc(r).size;
    a.dense = rc(t).nsons == 0 || cc(r).nsons == 0 ||
              (dense_small && std::min(m, n) <= DENSE_ACC_MIN && std::max(m, n) <= DENSE_ACC_MAX);
    a.R.cap = capof(m, n);
    return a;
  }

  void dense_ensure(SAcc& a) {
    if (a.dloc >= 0) return;
    int64_t m = rc(a.t).size, n = cc(a.r).size;
    int c = S.alloc(m * n);
    a.dhold = std::make_shared<Hold>(&S, c);
    a.dloc = S.chunk_loc(c);
    a.dld = (int)m;
    a.dobj = S.chunk_obj(c);
    HTask z = blank(T_ZERO);
    z.m = (int)m;
    z.n = (int)n;
    z.c = a.dloc;
    z.ldc = (int)m;
    S.emit(z, {}, {a.dobj});
    a.dzero = true;
  }

  // give a low-rank matrix its own storage (m x cap, n x cap) and rank slot
  void own_storage(SLow& L, int64_t m, int64_t n) {
    if (L.own) return;
    int c = S.alloc((m + n) * L.cap);
    L.hold = std::make_shared<Hold>(&S, c);
    L.u = S.chunk_loc(c);
    L.v = L.u + m * L.cap;
    L.ldu = (int)m;
    L.ldv = (int)n;
    L.obj = S.chunk_obj(c);
    L.own = true;
    L.slot = S.new_slot();
    L.wmax = L.cap;
  }

  // low-rank target <- trunc(target + alpha P) by one T_RKADD, in place.
  void rkadd_into(double alpha, const SProd& P, SLow& Z, int64_t m, int64_t n, int ft, int fr) {
    int rin = Z.zero ? -1 : (Z.wcode < 0 ? -(Z.wcode + 1) : -2);
    if (rin == -2) throw HmError(HMAT_ERR_INTERNAL, "rkadd: fixed-width target");
    int64_t cu = Z.u, cv = Z.v;
    int ldcu = Z.ldu, ldcv = Z.ldv, inobj = Z.obj;
    own_storage(Z, m, n);
    HTask t = blank(T_RKADD);
    t.flags = (P.aid ? F_A_IDENT : 0) | (P.bid ? F_B_IDENT : 0) | (P.btr ? F_B_TRANS : 0) | F_CHECK_ZERO;
    t.m = (int)m;
    t.n = (int)n;
    t.alpha = alpha;
    t.a = P.a;
    t.lda = P.lda;
    t.b = P.b;
    t.ldb = P.ldb;
    t.wa = P.wcode;
    t.c = rin >= 0 ? cu : -1;
    t.d = rin >= 0 ? cv : -1;
    t.ldc = ldcu;
    t.ldd = ldcv;
    t.rin = rin;
    t.e = Z.u;
    t.f = Z.v;
    t.lde = Z.ldu;
    t.ldf = Z.ldv;
    t.rout = Z.slot;
    t.cap = Z.cap;
    int64_t l = (int64_t)P.wcap + (rin >= 0 ? Z.wmax : 0);
    if (l > HM_LMAX_HOST) throw HmError(HMAT_ERR_RANK, "stacked width exceeds the truncation limit");
    int inmax = Z.wmax;
    // a large factored block of the mixed form: a gang of CTAs (TSQR)
    int G = 1;
    if (mixed && !P.aid && !P.bid && std::min(m, n) >= 4 * HM_GANG_MIN_ROWS && l <= 128)
      G = (int)std::min<int64_t>(8, std::min(m, n) / HM_GANG_MIN_ROWS);
    int64_t base_ws = rk_ws(m, n, l) + (mixed ? rand_ws(m, n, l) : 0);
    int ws = S.alloc(base_ws + (G > 1 ? gang_ws_doubles(m, n, l, G) : 0));
    t.ws = S.chunk_loc(ws);
    if (G > 1) {
      t.pad0 = 0;
      t.pad1 = G;
      t.q = (int)l;
      t.list_begin = (int32_t)base_ws;
    }
    std::vector<int> reads = P.objs;
    if (rin >= 0 && inobj >= 0 && inobj != Z.obj) reads.push_back(inobj);
    int32_t id0 = S.emit(t, reads, {Z.obj, S.chunk_obj(ws)});
    set_features(ft, fr);
    if (G > 1) S.emit_gang_members(id0, G);
    S.release(ws);
    Z.wcode = width_from_slot(Z.slot);
    Z.zero = false;
    Z.wmax = Z.cap;
    (void)inmax;
  }

  // C (m x n at cloc, ldc) += alpha Ahat Bhat^T of a product in low-rank
  // form, exactly (Fig. rkupdate, dense target).
  void dense_update(double alpha, const SProd& P, int64_t m, int64_t n, int64_t cloc, int ldc, int cobj) {
    if (P.aid && P.btr) throw HmError(HMAT_ERR_INTERNAL, "dense update: transposed identity product");
    HTask t = blank(P.aid || P.bid ? T_ADD : T_GEMM);
    t.m = (int)m;
    t.n = (int)n;
    t.alpha = alpha;
    t.c = cloc;
    t.ldc = ldc;
    if (P.aid) {
      t.flags = F_TRANS;  // C += alpha Bhat^T
      t.a = P.b;
      t.lda = P.ldb;
    } else if (P.bid) {
      t.a = P.a;
      t.lda = P.lda;
    } else {
      t.a = P.a;
      t.lda = P.lda;
      t.b = P.b;
      t.ldb = P.ldb;
      t.wa = P.wcode;
      t.flags = P.btr ? F_B_TRANS : 0;
    }
    std::vector<int> reads = P.objs;
    S.emit(t, reads, {cobj});
  }

  void add_product(double alpha, SProd& P, SAcc& a) {
    int64_t m = rc(a.t).size, n = cc(a.r).size;
    if (a.dense) {
      dense_ensure(a);
      HTask t = blank(P.aid || P.bid ? T_ADD : T_GEMM);
      t.m = (int)m;
      t.n = (int)n;
      t.alpha = alpha;
      t.c = a.dloc;
      t.ldc = a.dld;
      if (P.aid) {
        t.flags = F_TRANS;  // D += alpha Bhat^T
        t.a = P.b;
        t.lda = P.ldb;
      } else if (P.bid) {
        t.a = P.a;
        t.lda = P.lda;
      } else {
        t.a = P.a;
        t.lda = P.lda;
        t.b = P.b;
        t.ldb = P.ldb;
        t.wa = P.wcode;
        t.flags = P.btr ? F_B_TRANS : 0;
      }
      std::vector<int> reads = P.objs;
      S.emit(t, reads, {a.dobj});
      a.dzero = false;
    } else {
      rkadd_into(alpha, P, a.R, m, n, a.t, a.r);
    }
  }

  // Fig. addproduct
  void addproduct(double alpha, const hmat* X, int xb, const hmat* Y, int yb, SAcc& a) {
    if (X->kind(xb) != 0 || Y->kind(yb) != 0) {
      SProd P = leaf_product(X, xb, Y, yb);
      if (P.zero) return;
      add_product(alpha, P, a);
    } else {
      a.P.push_back(SPend{alpha, X, xb, Y, yb});
    }
  }

  // Fig. split
  std::vector<std::vector<SAcc>> split(SAcc& a) {
    const CNodeH& t = rc(a.t);
    const CNodeH& r = cc(a.r);
    std::vector<std::vector<SAcc>> sons((size_t)t.nsons);
    for (int i = 0; i < t.nsons; ++i)
      for (int j = 0; j < r.nsons; ++j) {
        SAcc s = acc_new(t.son[i], r.son[j]);
        int64_t ro = rc(s.t).off - t.off, co = cc(s.r).off - r.off;
        int64_t sm = rc(s.t).size, sn = cc(s.r).size;
        if (a.dense) {
          // the son's block of the parent's dense block: a view (or, while
          // the parent has no storage yet, a zero block of its own)
          s.dense = true;
          if (a.dloc >= 0) {
            s.dloc = a.dloc + ro + co * a.dld;
            s.dld = a.dld;
            s.dobj = a.dobj;
            s.dhold = a.dhold;
            s.dzero = a.dzero;
          }
        } else if (!a.R.zero) {
          if (s.dense) {
            dense_ensure(s);
            HTask g = blank(T_GEMM);
            g.flags = F_ZERO_OUT;
            g.m = (int)sm;
            g.n = (int)sn;
            g.alpha = 1.0;
            g.a = a.R.u + ro;
            g.lda = a.R.ldu;
            g.b = a.R.v + co;
            g.ldb = a.R.ldv;
            g.wa = a.R.wcode;
            g.c = s.dloc;
            g.ldc = s.dld;
            S.emit(g, {a.R.obj}, {s.dobj});
            s.dzero = false;
          } else {
            s.R = a.R;  // view
            s.R.own = false;
            s.R.u = a.R.u + ro;
            s.R.v = a.R.v + co;
            s.R.cap = capof(sm, sn);
          }
        }
        for (const SPend& p : a.P) {
          int ns = p.X->sc(p.xb).nsons;
          for (int k = 0; k < ns; ++k)
            addproduct(p.alpha, p.X, p.X->bt->child(p.xb, i, k), p.Y, p.Y->bt->child(p.yb, k, j), s);
        }
        sons[(size_t)i].push_back(std::move(s));
      }
    return sons;
  }

  // rkupdate of a factorised Rhat (Fig. rkupdate)
  void rkupdate(const SLow& R, int t, int r, STarget z) {
    if (R.zero) return;
    int64_t m = rc(t).size, n = cc(r).size;
    if (z.tmp) {
      SProd P;
      P.a = R.u;
      P.lda = R.ldu;
      P.b = R.v;
      P.ldb = R.ldv;
      P.wcode = R.wcode;
      P.wcap = R.wmax;
      P.objs.push_back(R.obj);
      rkadd_into(1.0, P, *z.tmp, m, n, t, r);
      return;
    }
    hmat* M = z.M;
    int kind = M->kind(z.b);
    if (kind == 1) {
      HTask g = blank(T_GEMM);
      g.m = (int)m;
      g.n = (int)n;
      g.alpha = 1.0;
      g.a = R.u;
      g.lda = R.ldu;
      g.b = R.v;
      g.ldb = R.ldv;
      g.wa = R.wcode;
      g.c = hl(M, z.b);
      g.ldc = (int)m;
      int o = obj_of(M, z.b);
      S.emit(g, {R.obj}, {o});
      M->zero[(size_t)z.b] = 0;
    } else if (kind == 2) {
      SLow L = leaf_low(M, z.b);
      SProd P;
      P.a = R.u;
      P.lda = R.ldu;
      P.b = R.v;
      P.ldb = R.ldv;
      P.wcode = R.wcode;
      P.wcap = R.wmax;
      P.objs.push_back(R.obj);
      rkadd_into(1.0, P, L, m, n, t, r);
      M->zero[(size_t)z.b] = 0;
    } else {
      const BNodeH& nd = M->bt->nodes[(size_t)z.b];
      const CNodeH& tt = rc(t);
      const CNodeH& rr = cc(r);
      for (int i = 0; i < tt.nsons; ++i)
        for (int j = 0; j < rr.nsons; ++j) {
          SLow V = R;
          V.u = R.u + (rc(tt.son[i]).off - tt.off);
          V.v = R.v + (cc(rr.son[j]).off - rr.off);
          STarget c;
          c.M = M;
          c.b = M->bt->child(z.b, i, j);
          c.t = tt.son[i];
          c.r = rr.son[j];
          (void)nd;
          rkupdate(V, c.t, c.r, c);
        }
    }
  }

  // low-rank leaf of an H-matrix as an SLow with its own storage and slot
  SLow leaf_low(hmat* M, int b) {
    SLow L;
    L.u = hl(M, b);
    L.v = hv(M, b);
    L.ldu = (int)M->rows(b);
    L.ldv = (int)M->cols(b);
    L.cap = M->cap[(size_t)b];
    L.slot = sl(M, b);
    L.wcode = width_from_slot(L.slot);
    L.obj = obj_of(M, b);
    L.own = true;
    L.zero = M->zero[(size_t)b];
    L.wmax = L.cap;
    return L;
  }

  // Block (t, r) of Z is a low-rank leaf (or a temporary) while the update
  // is finer: four temporaries, row-restricted views of Z's factors, receive
  // the updates of the sons through fill(i, j, target); then Fig. rkmerge
  // (rowmerge of the block columns, then of the row) writes the merged
  // result back (Fig. flush, third case; the standard multiplication does
  // the same).
  template <class F>
  void via_temporaries(int tcl, int rcl, STarget z, F fill) {
    if (!z.tmp && z.M->kind(z.b) != 2) throw HmError(HMAT_ERR_INTERNAL, "temporaries: dense target");
    SLow base = z.tmp ? *z.tmp : leaf_low(z.M, z.b);
    const CNodeH& tt = rc(tcl);
    const CNodeH& rr = cc(rcl);
    int64_t m = tt.size, n = rr.size;
    if (tt.nsons != 2 || rr.nsons != 2) throw HmError(HMAT_ERR_ARG, "rkmerge needs binary cluster trees");
    SLow tmp[2][2];
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) {
        SLow& T = tmp[i][j];
        T = base;
        T.own = false;
        T.u = base.u + (rc(tt.son[i]).off - tt.off);
        T.v = base.v + (cc(rr.son[j]).off - rr.off);
        T.cap = capof(rc(tt.son[i]).size, cc(rr.son[j]).size);
        T.hold = base.hold;
      }
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) {
        STarget c;
        c.tmp = &tmp[i][j];
        c.t = tt.son[i];
        c.r = rr.son[j];
        fill(i, j, c);
      }
    // Fig. rkmerge: merge the block columns (rowmerge of adjoints), then the row
    SLow col[2];
    for (int j = 0; j < 2; ++j) {
      int64_t nrj = cc(rr.son[j]).size;
      SLow& C = col[j];
      C.cap = capof(nrj, m);
      own_storage(C, nrj, m);  // "A" role: r_j x cap, "B" role: t x cap
      HTask t = blank(T_ROWMERGE);
      t.m = (int)nrj;
      t.p = (int)rc(tt.son[0]).size;
      t.q = (int)rc(tt.son[1]).size;
      t.a = tmp[0][j].v;
      t.lda = tmp[0][j].ldv;
      t.b = tmp[0][j].u;
      t.ldb = tmp[0][j].ldu;
      t.wa = tmp[0][j].zero ? 0 : tmp[0][j].wcode;
      t.c = tmp[1][j].v;
      t.ldc = tmp[1][j].ldv;
      t.d = tmp[1][j].u;
      t.ldd = tmp[1][j].ldu;
      t.wb = tmp[1][j].zero ? 0 : tmp[1][j].wcode;
      t.e = C.u;
      t.lde = C.ldu;
      t.f = C.v;
      t.ldf = C.ldv;
      t.rout = C.slot;
      t.cap = C.cap;
      int64_t l = (tmp[0][j].zero ? 0 : tmp[0][j].wmax) + (tmp[1][j].zero ? 0 : tmp[1][j].wmax);
      if (l > HM_LMAX_HOST) throw HmError(HMAT_ERR_RANK, "merged width exceeds the truncation limit");
      int64_t base_ws = rk_ws(nrj, m, l) + (int64_t)nrj * l + (mixed ? m * l + rand_ws(nrj, m, l) : 0);
      int G = merge_gang(nrj, (int64_t)t.p + t.q, l);
      int ws = S.alloc(base_ws + (G > 1 ? gang_ws_doubles(nrj, (int64_t)t.p + t.q, l, G) : 0));
      t.ws = S.chunk_loc(ws);
      std::vector<int> reads;
      for (int i = 0; i < 2; ++i)
        if (tmp[i][j].obj >= 0) reads.push_back(tmp[i][j].obj);
      int32_t id0 = S.emit(t, reads, {C.obj, S.chunk_obj(ws)});
      set_features(tcl, rr.son[j]);
      if (G > 1) make_merge_gang(id0, G, l, base_ws);
      S.release(ws);
      C.wcode = width_from_slot(C.slot);
      C.zero = false;
    }
    SLow out = base;
    if (z.tmp) {
      own_storage(*z.tmp, m, n);
      out = *z.tmp;
    }
    HTask t = blank(T_ROWMERGE);
    t.m = (int)m;
    t.p = (int)cc(rr.son[0]).size;
    t.q = (int)cc(rr.son[1]).size;
    t.a = col[0].v;  // column j = Bc_j Ac_j^T: "A" role Bc_j (t x k), "B" role Ac_j (r_j x k)
    t.lda = col[0].ldv;
    t.b = col[0].u;
    t.ldb = col[0].ldu;
    t.wa = col[0].wcode;
    t.c = col[1].v;
    t.ldc = col[1].ldv;
    t.d = col[1].u;
    t.ldd = col[1].ldu;
    t.wb = col[1].wcode;
    t.e = out.u;
    t.lde = out.ldu;
    t.f = out.v;
    t.ldf = out.ldv;
    t.rout = out.slot;
    t.cap = out.cap;
    int64_t l = (int64_t)col[0].cap + col[1].cap;
    if (l > HM_LMAX_HOST) throw HmError(HMAT_ERR_RANK, "merged width exceeds the truncation limit");
    int64_t base_ws = rk_ws(m, n, l) + (int64_t)m * l + (mixed ? n * l + rand_ws(m, n, l) : 0);
    int G = merge_gang(m, (int64_t)t.p + t.q, l);
    int ws = S.alloc(base_ws + (G > 1 ? gang_ws_doubles(m, (int64_t)t.p + t.q, l, G) : 0));
    t.ws = S.chunk_loc(ws);
    int32_t id0 = S.emit(t, {col[0].obj, col[1].obj}, {out.obj, S.chunk_obj(ws)});
    set_features(tcl, rcl);
    if (G > 1) make_merge_gang(id0, G, l, base_ws);
    S.release(ws);
    if (z.tmp) {
      z.tmp->wcode = width_from_slot(z.tmp->slot);
      z.tmp->zero = false;
    } else {
      z.M->zero[(size_t)z.b] = 0;
    }
  }

  // The pending products of a dense accumulator expanded down to the leaf
  // cases, each added exactly into the accumulator's own block (its sons are
  // views of it; Fig. split with the son accumulators in the parent's block).
  void resolve_pending(SAcc& a) {
    auto sons = split(a);
    for (auto& row : sons)
      for (SAcc& c : row)
        if (!c.P.empty()) resolve_pending(c);
    a.P.clear();
  }

  // Fig. flush
  void flush(SAcc& a, STarget z) {
    int64_t m = rc(a.t).size, n = cc(a.r).size;
    if (a.dense) {
      if (!z.tmp && z.M->kind(z.b) == 0) {
        // subdivided target: the sub-blocks (and the pending products split
        // over them) into the sons of the target
        auto sons = split(a);
        for (size_t i = 0; i < sons.size(); ++i)
          for (size_t j = 0; j < sons[i].size(); ++j)
            flush(sons[i][j], target_of(z.M, z.M->bt->child(z.b, (int)i, (int)j), sons[i][j].t, sons[i][j].r));
        a.P.clear();
        a.dhold.reset();
        a.dloc = -1;
        a.dzero = true;
        return;
      }
      if (!a.P.empty()) {
        // a leaf target: every pending product added into the block itself
        dense_ensure(a);
        resolve_pending(a);
        a.dzero = false;
      }
      if (a.dloc < 0 || a.dzero) return;
      bool zdense = !z.tmp && z.M->kind(z.b) == 1;
      if (zdense) {
        HTask t = blank(T_ADD);
        t.m = (int)m;
        t.n = (int)n;
        t.alpha = 1.0;
        t.a = a.dloc;
        t.lda = a.dld;
        t.c = hl(z.M, z.b);
        t.ldc = (int)m;
        int o = obj_of(z.M, z.b);
        S.emit(t, {a.dobj}, {o});
        z.M->zero[(size_t)z.b] = 0;
      } else {
        if (!z.tmp && z.M->kind(z.b) != 2) throw HmError(HMAT_ERR_INTERNAL, "flush: dense accumulator, subdivided target");
        SProd P;
        P.objs.push_back(a.dobj);
        if (m <= n) {
          P.aid = true;
          P.b = a.dloc;
          P.ldb = a.dld;
          P.btr = true;
          P.wcode = P.wcap = (int)m;
        } else {
          P.bid = true;
          P.a = a.dloc;
          P.lda = a.dld;
          P.wcode = P.wcap = (int)n;
        }
        if (z.tmp) {
          rkadd_into(1.0, P, *z.tmp, m, n, a.t, a.r);
        } else {
          SLow L = leaf_low(z.M, z.b);
          rkadd_into(1.0, P, L, m, n, a.t, a.r);
          z.M->zero[(size_t)z.b] = 0;
        }
      }
      a.P.clear();
      a.dhold.reset();
      a.dloc = -1;
      a.dzero = true;
      return;
    }
    if (a.P.empty()) {
      rkupdate(a.R, a.t, a.r, z);
    } else if (!z.tmp && z.M->kind(z.b) == 0) {
      auto sons = split(a);
      for (size_t i = 0; i < sons.size(); ++i)
        for (size_t j = 0; j < sons[i].size(); ++j) {
          STarget c;
          c.M = z.M;
          c.b = z.M->bt->child(z.b, (int)i, (int)j);
          c.t = sons[i][j].t;
          c.r = sons[i][j].r;
          flush(sons[i][j], c);
        }
    } else {
      // (t, r) is a leaf of Z with pending products: temporaries + rkmerge
      auto sons = split(a);
      via_temporaries(a.t, a.r, z, [&](int i, int j, STarget c) { flush(sons[(size_t)i][(size_t)j], c); });
    }
    a.P.clear();
    a.R = SLow();
  }

  // ---- standard multiplication (Section 4 before "Accumulated updates") ------
  // The product P of a leaf pair restricted to rows ro.. (rn of them) of its
  // row cluster and columns co.. (cn) of its column cluster: row ranges of
  // the factors; an identity factor becomes a block of the dense one
  // (Section 3, "Splitting": no arithmetic).
  SProd restrict_prod(const SProd& P, int64_t ro, int64_t rn, int64_t co, int64_t cn) const {
    SProd Q = P;
    if (P.aid) {  // A = I, Bhat^T given (m x n): block (t', r') of Bhat^T, A = I
      Q.b = P.btr ? P.b + ro + co * P.ldb : P.b + co + ro * P.ldb;
      Q.wcode = Q.wcap = (int)rn;
    } else if (P.bid) {  // B = I, Ahat (m x n): block (t', r') of Ahat
      Q.a = P.a + ro + co * P.lda;
      Q.wcode = Q.wcap = (int)cn;
    } else {
      Q.a = P.a + ro;
      Q.b = P.btr ? P.b + co * P.ldb : P.b + co;
    }
    return Q;
  }

  // Fig. rkupdate of alpha P into the block (t, r) of Z (or a temporary):
  // dense leaf N += alpha Ahat Bhat^T, admissible leaf rkadd (one truncation
  // per product), subdivided block the product restricted to the sons.
  void rkupdate_prod(double alpha, const SProd& P, int t, int r, STarget z) {
    int64_t m = rc(t).size, n = cc(r).size;
    if (z.tmp) {
      rkadd_into(alpha, P, *z.tmp, m, n, t, r);
      return;
    }
    hmat* M = z.M;
    int kind = M->kind(z.b);
    if (kind == 1) {
      dense_update(alpha, P, m, n, hl(M, z.b), (int)m, obj_of(M, z.b));
      M->zero[(size_t)z.b] = 0;
    } else if (kind == 2) {
      SLow L = leaf_low(M, z.b);
      rkadd_into(alpha, P, L, m, n, t, r);
      M->zero[(size_t)z.b] = 0;
    } else {
      const CNodeH& tt = rc(t);
      const CNodeH& rr = cc(r);
      for (int i = 0; i < tt.nsons; ++i)
        for (int j = 0; j < rr.nsons; ++j) {
          const CNodeH& ti = rc(tt.son[i]);
          const CNodeH& rj = cc(rr.son[j]);
          SProd Q = restrict_prod(P, ti.off - tt.off, ti.size, rj.off - rr.off, rj.size);
          rkupdate_prod(alpha, Q, tt.son[i], rr.son[j], target_of(M, M->bt->child(z.b, i, j), tt.son[i], rr.son[j]));
        }
    }
  }

  // Z|_{t x r} <- Z|_{t x r} + alpha X|_{t x s} Y|_{s x r} with every product
  // of a leaf pair applied at once (the standard form the accumulated one is
  // compared with; Section 4, the remark after the complexity theorem).
  void mult_std(double alpha, const hmat* X, int xb, const hmat* Y, int yb, STarget z) {
    if (X->kind(xb) != 0 || Y->kind(yb) != 0) {
      SProd P = leaf_product(X, xb, Y, yb);
      if (!P.zero) rkupdate_prod(alpha, P, z.t, z.r, z);
      return;
    }
    int ns = X->sc(xb).nsons;
    if (!z.tmp && z.M->kind(z.b) == 0) {
      const CNodeH& tt = rc(z.t);
      const CNodeH& rr = cc(z.r);
      for (int i = 0; i < tt.nsons; ++i)
        for (int j = 0; j < rr.nsons; ++j) {
          STarget c = target_of(z.M, z.M->bt->child(z.b, i, j), tt.son[i], rr.son[j]);
          for (int k = 0; k < ns; ++k) mult_std(alpha, X, X->bt->child(xb, i, k), Y, Y->bt->child(yb, k, j), c);
        }
      return;
    }
    // (t, r) is a leaf of Z (or a temporary) and the product is finer
    via_temporaries(z.t, z.r, z, [&](int i, int j, STarget c) {
      for (int k = 0; k < ns; ++k) mult_std(alpha, X, X->bt->child(xb, i, k), Y, Y->bt->child(yb, k, j), c);
    });
  }

  // ---- H-LU in the standard form ---------------------------------------------
  void trsm_L_std(hmat* G, int d, int b) {
    if (G->kind(b) != 0) {
      trsm_L(G, d, b);  // leaf: the same H-solve as the accumulated form
      return;
    }
    const CNodeH& t = G->tc(b);
    const CNodeH& r = G->sc(b);
    for (int j = 0; j < r.nsons; ++j)
      for (int i = 0; i < t.nsons; ++i) {
        int bi = G->bt->child(b, i, j);
        trsm_L_std(G, G->bt->child(d, i, i), bi);
        for (int l = i + 1; l < t.nsons; ++l)
          mult_std(-1.0, G, G->bt->child(d, l, i), G, bi, target_of(G, G->bt->child(b, l, j), t.son[l], r.son[j]));
      }
  }

  void trsm_U_std(hmat* G, int d, int b) {
    if (G->kind(b) != 0) {
      trsm_U(G, d, b);
      return;
    }
    const CNodeH& r = G->tc(b);
    const CNodeH& t = G->sc(b);
    for (int j = 0; j < r.nsons; ++j)
      for (int i = 0; i < t.nsons; ++i) {
        int bi = G->bt->child(b, j, i);
        trsm_U_std(G, G->bt->child(d, i, i), bi);
        for (int l = i + 1; l < t.nsons; ++l)
          mult_std(-1.0, G, bi, G, G->bt->child(d, i, l), target_of(G, G->bt->child(b, j, l), r.son[j], t.son[l]));
      }
  }

  // Block LU with Schur complement (Section 6) with every update applied at
  // once.
  void lu_std(hmat* G, int b) {
    int kind = G->kind(b);
    if (kind == 1) {
      HTask t = blank(T_LU);
      t.m = (int)G->rows(b);
      t.a = hl(G, b);
      t.lda = t.m;
      S.emit(t, {}, {obj_of(G, b)});
      return;
    }
    if (kind != 0) throw HmError(HMAT_ERR_ARG, "H-LU: admissible diagonal block");
    const CNodeH& t = G->tc(b);
    int p = t.nsons;
    for (int i = 0; i < p; ++i) {
      int di = G->bt->child(b, i, i);
      lu_std(G, di);
      for (int j = i + 1; j < p; ++j) trsm_L_std(G, di, G->bt->child(b, i, j));
      for (int j = i + 1; j < p; ++j) trsm_U_std(G, di, G->bt->child(b, j, i));
      for (int j = i + 1; j < p; ++j)
        for (int l = i + 1; l < p; ++l)
          mult_std(-1.0, G, G->bt->child(b, j, i), G, G->bt->child(b, i, l),
                   target_of(G, G->bt->child(b, j, l), t.son[j], t.son[l]));
    }
  }

  // ---- H-LU with accumulators --------------------------------------------------
  void trsm_L(hmat* G, int d, int b) {
    int kind = G->kind(b);
    if (kind == 1) {
      if (!G->zero[(size_t)b])
        hsolve(G, d, TRSM_L, hl(G, b), (int)G->rows(b), obj_of(G, b), (int)G->cols(b));
    } else if (kind == 2) {
      if (!G->zero[(size_t)b])
        hsolve(G, d, TRSM_L, hl(G, b), (int)G->rows(b), obj_of(G, b), width_from_slot(sl(G, b)));
    } else {
      const CNodeH& t = G->tc(b);
      const CNodeH& r = G->sc(b);
      for (int j = 0; j < r.nsons; ++j) {
        std::vector<SAcc> acc;
        for (int i = 0; i < t.nsons; ++i) acc.push_back(acc_new(t.son[i], r.son[j]));
        for (int i = 0; i < t.nsons; ++i) {
          int bi = G->bt->child(b, i, j);
          STarget z;
          z.M = G;
          z.b = bi;
          z.t = t.son[i];
          z.r = r.son[j];
          flush(acc[(size_t)i], z);
          trsm_L(G, G->bt->child(d, i, i), bi);
          for (int l = i + 1; l < t.nsons; ++l) addproduct(-1.0, G, G->bt->child(d, l, i), G, bi, acc[(size_t)l]);
        }
      }
    }
  }

  void trsm_U(hmat* G, int d, int b) {
    int kind = G->kind(b);
    if (kind == 1) {
      if (G->zero[(size_t)b]) return;
      // X U = N  <=>  U^T X^T = N^T: solve on a transposed copy
      int m = (int)G->rows(b), n = (int)G->cols(b);
      int c = S.alloc((int64_t)m * n);
      int cobj = S.chunk_obj(c);
      int bobj = obj_of(G, b);
      HTask t1 = blank(T_COPY);
      t1.flags = F_TRANS;
      t1.m = n;
      t1.n = m;
      t1.a = hl(G, b);
      t1.lda = m;
      t1.c = S.chunk_loc(c);
      t1.ldc = n;
      S.emit(t1, {bobj}, {cobj});
      hsolve(G, d, TRSM_UT, S.chunk_loc(c), n, cobj, m);
      HTask t2 = blank(T_COPY);
      t2.flags = F_TRANS;
      t2.m = m;
      t2.n = n;
      t2.a = S.chunk_loc(c);
      t2.lda = n;
      t2.c = hl(G, b);
      t2.ldc = m;
      S.emit(t2, {cobj}, {bobj});
      S.release(c);
    } else if (kind == 2) {
      if (!G->zero[(size_t)b])
        hsolve(G, d, TRSM_UT, hv(G, b), (int)G->cols(b), obj_of(G, b),
               width_from_slot(sl(G, b)));
    } else {
      const CNodeH& r = G->tc(b);
      const CNodeH& t = G->sc(b);
      for (int j = 0; j < r.nsons; ++j) {
        std::vector<SAcc> acc;
        for (int i = 0; i < t.nsons; ++i) acc.push_back(acc_new(r.son[j], t.son[i]));
        for (int i = 0; i < t.nsons; ++i) {
          int bi = G->bt->child(b, j, i);
          STarget z;
          z.M = G;
          z.b = bi;
          z.t = r.son[j];
          z.r = t.son[i];
          flush(acc[(size_t)i], z);
          trsm_U(G, G->bt->child(d, i, i), bi);
          for (int l = i + 1; l < t.nsons; ++l) addproduct(-1.0, G, bi, G, G->bt->child(d, i, l), acc[(size_t)l]);
        }
      }
    }
  }

  // ---- H-Cholesky with accumulated updates -----------------------------------
  // M's block dst (s x t) <- block src (t x s) transposed, leaf by leaf (the
  // block tree of one cluster tree is symmetric): dense leaves by a transposed
  // copy, low-rank leaves by swapping the factors and the rank.
  void transpose_block(hmat* M, int src, int dst) {
    const BNodeH& nd = M->bt->nodes[(size_t)src];
    if (nd.kind == 0) {
      int ns = M->tc(src).nsons, nr = M->sc(src).nsons;
      for (int i = 0; i < ns; ++i)
        for (int j = 0; j < nr; ++j) transpose_block(M, M->bt->child(src, i, j), M->bt->child(dst, j, i));
      return;
    }
    int m = (int)M->rows(src), n = (int)M->cols(src);
    if (nd.kind == 1) {
      HTask c = blank(T_COPY);
      c.flags = F_TRANS;
      c.m = n;
      c.n = m;
      c.a = hl(M, src);
      c.lda = m;
      c.c = hl(M, dst);
      c.ldc = n;
      S.emit(c, {obj_of(M, src)}, {obj_of(M, dst)});
    } else {
      int cap = M->cap[(size_t)src];
      HTask u = blank(T_COPY);  // U_dst (n x cap) <- V_src
      u.m = n;
      u.n = cap;
      u.a = hv(M, src);
      u.lda = n;
      u.c = hl(M, dst);
      u.ldc = n;
      S.emit(u, {obj_of(M, src)}, {obj_of(M, dst)});
      HTask v = blank(T_COPY);  // V_dst (m x cap) <- U_src
      v.m = m;
      v.n = cap;
      v.a = hl(M, src);
      v.lda = m;
      v.c = hv(M, dst);
      v.ldc = m;
      S.emit(v, {obj_of(M, src)}, {obj_of(M, dst)});
      HTask r = blank(T_RANKSET);
      r.rout = sl(M, dst);
      r.wa = -(sl(M, src) + 1);
      S.emit(r, {obj_of(M, src)}, {obj_of(M, dst)});
    }
    M->zero[(size_t)dst] = M->zero[(size_t)src];
  }

  // chol(t): chol(t1); flush the (2,1) updates and solve L21 = G21 L11^{-T}
  // (the LU's right solve, U = L11^T sits above the diagonal); mirror L21^T
  // into the (1,2) block; addproduct the Schur update -L21 L21^T without flush;
  // chol(t2) takes the accumulator.  The (1,2) accumulator is dropped: its
  // updates are the transposes of the (2,1) ones.
  void chol(hmat* G, int b, SAcc& acc) {
    int kind = G->kind(b);
    if (kind == 1) {
      STarget z;
      z.M = G;
      z.b = b;
      z.t = acc.t;
      z.r = acc.r;
      flush(acc, z);
      HTask t = blank(T_CHOL);
      t.m = (int)G->rows(b);
      t.a = hl(G, b);
      t.lda = t.m;
      S.emit(t, {}, {obj_of(G, b)});
      return;
    }
    if (kind != 0) throw HmError(HMAT_ERR_ARG, "H-Cholesky: admissible diagonal block");
    if (G->tc(b).nsons != 2) throw HmError(HMAT_ERR_ARG, "H-Cholesky: the cluster tree must be binary");
    int c1 = G->tc(b).son[0], c2 = G->tc(b).son[1];
    auto sub = split(acc);
    acc.P.clear();
    acc.R = SLow();
    int b11 = G->bt->child(b, 0, 0), b12 = G->bt->child(b, 0, 1);
    int b21 = G->bt->child(b, 1, 0), b22 = G->bt->child(b, 1, 1);
    chol(G, b11, sub[0][0]);
    STarget z;
    z.M = G;
    z.b = b21;
    z.t = c2;
    z.r = c1;
    flush(sub[1][0], z);
    trsm_U(G, b11, b21);
    transpose_block(G, b21, b12);
    addproduct(-1.0, G, b21, G, b12, sub[1][1]);
    chol(G, b22, sub[1][1]);
  }

  // ---- H-matrix inversion with accumulated updates (Fig. invert) -------------
  // Every leaf of M's subtree b set to zero (dense leaves zeroed, admissible
  // leaves rank 0), and marked structurally zero for the products that follow.
  void zero_leaves(hmat* M, int b) {
    const BNodeH& nd = M->bt->nodes[(size_t)b];
    if (nd.kind == 0) {
      for (int k = 0; k < nd.nsons; ++k) zero_leaves(M, M->bt->sons[(size_t)(nd.son0 + k)]);
      return;
    }
    if (M->zero[(size_t)b]) return;
    HTask z = blank(nd.kind == 1 ? T_ZERO : T_RANKSET);
    if (nd.kind == 1) {
      z.m = (int)M->rows(b);
      z.n = (int)M->cols(b);
      z.c = hl(M, b);
      z.ldc = z.m;
    } else {
      z.rout = sl(M, b);
      z.wa = 0;
    }
    S.emit(z, {}, {obj_of(M, b)});
    M->zero[(size_t)b] = 1;
  }

  STarget target_of(hmat* M, int b, int t, int r) {
    STarget z;
    z.M = M;
    z.b = b;
    z.t = t;
    z.r = r;
    return z;
  }

  // G|_{t x t} <- (G|_{t x t} + the updates pending in acc)^{-1}; H: auxiliary
  // storage of H_12, H_21 on the same block tree.  The six steps of Fig.
  // invert, with its last product accumulated for t_1 x t_1 and flushed into
  // G_11, and a fresh accumulator for every product that is flushed.
  void invert(hmat* G, hmat* H, int b, SAcc& acc) {
    int kind = G->kind(b);
    if (kind == 1) {
      flush(acc, target_of(G, b, acc.t, acc.r));
      HTask t = blank(T_INV);
      t.m = (int)G->rows(b);
      t.a = hl(G, b);
      t.lda = t.m;
      S.emit(t, {}, {obj_of(G, b)});
      G->zero[(size_t)b] = 0;
      return;
    }
    if (kind != 0) throw HmError(HMAT_ERR_ARG, "H-inverse: admissible diagonal block");
    if (G->tc(b).nsons != 2) throw HmError(HMAT_ERR_ARG, "H-inverse: the cluster tree must be binary");
    int c1 = G->tc(b).son[0], c2 = G->tc(b).son[1];
    auto sub = split(acc);
    acc.P.clear();
    acc.R = SLow();
    int b11 = G->bt->child(b, 0, 0), b12 = G->bt->child(b, 0, 1);
    int b21 = G->bt->child(b, 1, 0), b22 = G->bt->child(b, 1, 1);
    invert(G, H, b11, sub[0][0]);                                  // 1. G_11^{-1}
    flush(sub[0][1], target_of(G, b12, c1, c2));
    flush(sub[1][0], target_of(G, b21, c2, c1));
    zero_leaves(H, b12);
    zero_leaves(H, b21);
    {
      SAcc a = acc_new(c1, c2);                                    // 2. H_12 = G_11^{-1} G_12
      addproduct(1.0, G, b11, G, b12, a);
      flush(a, target_of(H, b12, c1, c2));
    }
    {
      SAcc a = acc_new(c2, c1);                                    //    H_21 = G_21 G_11^{-1}
      addproduct(1.0, G, b21, G, b11, a);
      flush(a, target_of(H, b21, c2, c1));
    }
    addproduct(-1.0, H, b21, G, b12, sub[1][1]);                  // 3. S = G_22 - H_21 G_12
    invert(G, H, b22, sub[1][1]);                                  // 4. S^{-1}
    zero_leaves(G, b12);
    zero_leaves(G, b21);
    {
      SAcc a = acc_new(c1, c2);                                    // 5. H_12' = -H_12 S^{-1}
      addproduct(-1.0, H, b12, G, b22, a);
      flush(a, target_of(G, b12, c1, c2));
    }
    {
      SAcc a = acc_new(c2, c1);                                    //    H_21' = -S^{-1} H_21
      addproduct(-1.0, G, b22, H, b21, a);
      flush(a, target_of(G, b21, c2, c1));
    }
    {
      SAcc a = acc_new(c1, c1);                                    // 6. H_11' = G_11^{-1} - H_12 H_21'
      addproduct(-1.0, H, b12, G, b21, a);
      flush(a, target_of(G, b11, c1, c1));
    }
  }

  void lu(hmat* G, int b, SAcc& acc) {
    int kind = G->kind(b);
    if (kind == 1) {
      STarget z;
      z.M = G;
      z.b = b;
      z.t = acc.t;
      z.r = acc.r;
      flush(acc, z);
      HTask t = blank(T_LU);
      t.m = (int)G->rows(b);
      t.a = hl(G, b);
      t.lda = t.m;
      int o = obj_of(G, b);
      S.emit(t, {}, {o});
      return;
    }
    if (kind != 0) throw HmError(HMAT_ERR_ARG, "H-LU: admissible diagonal block");
    auto sub = split(acc);
    acc.P.clear();
    acc.R = SLow();
    int p = G->tc(b).nsons;
    for (int i = 0; i < p; ++i) {
      int di = G->bt->child(b, i, i);
      lu(G, di, sub[(size_t)i][(size_t)i]);
      for (int j = i + 1; j < p; ++j) {
        int bij = G->bt->child(b, i, j);
        STarget z;
        z.M = G;
        z.b = bij;
        z.t = sub[(size_t)i][(size_t)j].t;
        z.r = sub[(size_t)i][(size_t)j].r;
        flush(sub[(size_t)i][(size_t)j], z);
        trsm_L(G, di, bij);
      }
      for (int j = i + 1; j < p; ++j) {
        int bji = G->bt->child(b, j, i);
        STarget z;
        z.M = G;
        z.b = bji;
        z.t = sub[(size_t)j][(size_t)i].t;
        z.r = sub[(size_t)j][(size_t)i].r;
        flush(sub[(size_t)j][(size_t)i], z);
        trsm_U(G, di, bji);
      }
      for (int j = i + 1; j < p; ++j)
        for (int l = i + 1; l < p; ++l)
          addproduct(-1.0, G, G->bt->child(b, j, i), G, G->bt->child(b, i, l), sub[(size_t)j][(size_t)l]);
    }
  }
};

// ===========================================================================
// Running a task list
// ===========================================================================
struct RunResult {
  int status = 0;
  double ms = 0.0;
  unsigned long long truncations = 0;
  double flops = 0.0;
  double flops32 = 0.0;
  double bytes = 0.0;  // algorithmic bytes of the tasks
  unsigned long long type_ns[16] = {0}, type_cnt[16] = {0}, wait_ns = 0;
  unsigned long long rand_ok = 0, rand_fail = 0, sketch_attempts = 0, sketch_cols = 0;
  unsigned long long bad[6] = {0, 0, 0, 0, 0, 0};
  long long fail_task = -1;  // task that recorded the device status first (-1: none)
  unsigned long long gang = 0;  // truncations run by a gang of CTAs
  std::vector<uint32_t> task_ns;  // filled when profiling
  std::vector<uint32_t> task_aux;
};

// HMAT_PROFILE_TASKS=1 records every task's duration and reports the
// measured critical path (longest chain of task durations) by task type;
// HMAT_PROFILE_PATH=<file> also writes that path, one task per line (CSV).
bool profile_tasks() {
  const char* v = std::getenv("HMAT_PROFILE_TASKS");
  return v && v[0] == '1';
}

void critical_path(const Sched& S, const std::vector<uint32_t>& ns, const std::vector<uint32_t>& aux,
                   hmat_stats& st) {
  size_t n = S.tasks.size();
  std::vector<double> fin(n, 0.0);
  std::vector<int32_t> from(n, -1);
  for (size_t i = 0; i < n; ++i) {
    double start = 0.0;
    for (int64_t k = S.dep_ptr[i]; k < S.dep_ptr[i + 1]; ++k) {
      int32_t d = S.dep_idx[(size_t)k];
      if (fin[(size_t)d] > start) {
        start = fin[(size_t)d];
        from[i] = d;
      }
    }
    fin[i] = start + ns[i] * 1e-9;
  }
  size_t last = 0;
  for (size_t i = 1; i < n; ++i)
    if (fin[i] > fin[last]) last = i;
  st.cp_seconds = n ? fin[last] : 0.0;
  for (int t = 0; t < 16; ++t) {
    st.cp_type_seconds[t] = 0.0;
    st.cp_type_count[t] = 0;
  }
  const char* dump = std::getenv("HMAT_PROFILE_PATH");
  FILE* f = dump ? std::fopen(dump, "w") : nullptr;
  if (f) std::fprintf(f, "task,type,m,n,p,cap,ns,finish_s,l,path,failed,k,attempts\n");
  for (int64_t i = n ? (int64_t)last : -1; i >= 0; i = from[(size_t)i]) {
    const HTask& t = S.tasks[(size_t)i];
    st.cp_type_seconds[t.type] += ns[(size_t)i] * 1e-9;
    st.cp_type_count[t.type] += 1;
    uint32_t a = aux.empty() ? 0u : aux[(size_t)i];
    if (f)
      std::fprintf(f, "%lld,%d,%d,%d,%d,%d,%u,%.9f,%u,%u,%u,%u,%u\n", (long long)i, t.type, t.m, t.n, t.p, t.cap,
                   ns[(size_t)i], fin[(size_t)i], a & 0xFFFu, (a >> 12) & 7u, (a >> 15) & 1u, (a >> 16) & 0xFFu,
                   a >> 24);
  }
  if (f) std::fclose(f);
}

const char* task_name(int type) {
  static const char* names[] = {"NOP", "leaf LU", "leaf TRSM", "H x thin dense", "densify", "GEMM", "add",
                                "rkadd", "rowmerge", "copy", "zero", "rankset", "leaf inverse", "leaf Cholesky"};
  return type >= 0 && type < 14 ? names[type] : "?";
}

// " in task i (kind, sizes)" and, for a dense diagonal leaf task, the
// block-tree node of that leaf: the context of a device status.
std::string describe_failure(const Sched& S, long long ft, hmat* const* Hs, int count, const double* base) {
  if (ft < 0 || ft >= (long long)S.tasks.size()) return "";
  const HTask& t = S.tasks[(size_t)ft];
  std::string out = " in task " + std::to_string(ft) + " (" + task_name(t.type) + ", " + std::to_string(t.m) + " x " +
                    std::to_string(t.type == T_LU || t.type == T_CHOL || t.type == T_INV ? t.m : t.n) + ")";
  if ((t.type == T_LU || t.type == T_CHOL || t.type == T_INV) && t.a >= 0 && ((t.a >> 60) & 3) == 0) {
    for (int i = 0; i < count; ++i) {
      int64_t hoff = (int64_t)(Hs[i]->store.as<double>() - base);
      for (size_t b = 0; b < Hs[i]->bt->nodes.size(); ++b)
        if (Hs[i]->kind((int)b) == 1 && Hs[i]->loc[b] + hoff == t.a) {
          const CNodeH& c = Hs[i]->tc((int)b);
          out += ": dense diagonal leaf, block-tree node " + std::to_string(b) + (count > 1 ? " of matrix " + std::to_string(i) : "") +
                 ", permuted rows " + std::to_string(c.off) + ".." + std::to_string(c.off + c.size - 1);
          return out;
        }
    }
  }
  return out;
}

// A schedule uploaded to the device, with its scratch arena.
struct DevSched {
  DevBuf tasks, ptr, idx, leaves, done, gang, ws, misc, tns, feat, rec;
  size_t ntasks = 0;
};

// What a launch needs beyond the schedule: the rank predictor and whether the
// exact truncations record training pairs.
struct LaunchOpts {
  const void* mlp = nullptr;
  bool record = false;
  std::vector<float>* rec_out = nullptr;
  uint64_t seed = 0;  // 0: the default seed of the randomised sketches
  int rank_rule = 0;  // HMAT_REL_FRO or HMAT_REL_SPEC
};

void upload_sched(hmat_ctx* ctx, const Sched& S, DevSched& D) {
  cudaStream_t st = ctx->stream;
  upload(D.tasks, S.tasks, st);
  upload(D.ptr, S.dep_ptr, st);
  upload(D.idx, S.dep_idx, st);
  upload(D.leaves, S.leaves, st);
  upload(D.feat, S.feat, st);
  D.done.alloc(S.tasks.size() * sizeof(int));
  D.gang.alloc(S.tasks.size() * sizeof(int));
  D.ws.alloc((size_t)std::max<int64_t>(S.ws_top, 1) * sizeof(double));
  D.misc.alloc(64 * 8);
  D.ntasks = S.tasks.size();
}

RunResult launch_sched(hmat_ctx* ctx, const Sched& S, DevSched& D, double* hbase, int* ranks, double eps,
                       int64_t spin_limit, double* ext0, double* ext1, bool mixed, const LaunchOpts& lo = LaunchOpts()) {
  RunResult rr;
  if (D.ntasks == 0) return rr;
  cudaStream_t st = ctx->stream;
  HM_CUDA(cudaMemsetAsync(D.done.p, 0, D.ntasks * sizeof(int), st));
  HM_CUDA(cudaMemsetAsync(D.gang.p, 0, D.ntasks * sizeof(int), st));
  HM_CUDA(cudaMemsetAsync(D.misc.p, 0, 64 * 8, st));
  ExecEnv e;
  e.hbase = hbase;
  e.wsbase = D.ws.as<double>();
  e.ext0 = ext0;
  e.ext1 = ext1;
  e.ranks = ranks;
  e.tasks = D.tasks.as<HTask>();
  e.ntasks = (long long)D.ntasks;
  e.dep_ptr = D.ptr.as<int64_t>();
  e.dep_idx = D.idx.as<int32_t>();
  e.leaves = D.leaves.as<LeafRef>();
  e.done = D.done.as<int>();
  e.gang = D.gang.as<int>();
  void* dmp = D.misc.p;
  e.head = (unsigned long long*)dmp;
  e.counters = (unsigned long long*)dmp + 44;
  e.status = (int*)((unsigned long long*)dmp + 2);
  e.fail_task = (long long*)dmp + 5;
  e.flops = (double*)((unsigned long long*)dmp + 3);
  e.flops32 = (double*)((unsigned long long*)dmp + 4);
  e.bytes = (double*)((unsigned long long*)dmp + 6);
  e.type_ns = (unsigned long long*)dmp + 8;
  e.type_cnt = (unsigned long long*)dmp + 24;
  e.wait_ns = (unsigned long long*)dmp + 40;
  e.task_ns = nullptr;
  e.task_aux = nullptr;
  if (profile_tasks()) {
    D.tns.alloc(2 * D.ntasks * sizeof(uint32_t));
    HM_CUDA(cudaMemsetAsync(D.tns.p, 0, 2 * D.ntasks * sizeof(uint32_t), st));
    e.task_ns = D.tns.as<uint32_t>();
    e.task_aux = e.task_ns + D.ntasks;
  }
  e.feat = D.feat.as<float>();
  e.mlp = lo.mlp;
  e.oversample = 3;
  e.rec = nullptr;
  e.rec_count = (unsigned long long*)dmp + 60;
  e.rec_cap = 0;
  if (lo.record) {
    e.rec_cap = (long long)std::max<size_t>(D.ntasks / 2, 1024);
    D.rec.alloc((size_t)e.rec_cap * 7 * sizeof(float));
    e.rec = D.rec.as<float>();
  }
  e.eps = eps;
  e.rank_rule = lo.rank_rule;
  e.mixed = mixed ? 1 : 0;
  e.rand_min_l = 8;
  e.seed = lo.seed ? lo.seed : 0x5EEDull;
  e.spin_iters = spin_limit > 0 ? spin_limit : (1ll << 28);
  e.spin_ns = 20ull * 1000000000ull;
  // One CTA per SM when the schedule's average parallelism (estimated work
  // over its critical path) cannot keep two per SM busy: co-resident CTAs
  // then only slow the critical path down (they share the SM's pipes).
  int bps = ctx->blocks_per_sm;
  double cp = S.critical_flops();
  if (bps > 1 && cp > 0.0 && S.est_total < 2.0 * ctx->num_sms * cp) bps = 1;
  int grid = ctx->num_sms * bps;
  cudaEvent_t e0, e1;
  HM_CUDA(cudaEventCreate(&e0));
  HM_CUDA(cudaEventCreate(&e1));
  HM_CUDA(cudaEventRecord(e0, st));
  HM_CUDA(launch_exec(e, grid, st));
  HM_CUDA(cudaEventRecord(e1, st));
  unsigned long long misc[64];
  HM_CUDA(cudaMemcpyAsync(misc, dmp, sizeof(misc), cudaMemcpyDeviceToHost, st));
  HM_CUDA(cudaStreamSynchronize(st));
  for (int i = 0; i < 16; ++i) {
    rr.type_ns[i] = misc[8 + i];
    rr.type_cnt[i] = misc[24 + i];
  }
  rr.wait_ns = misc[40];
  float ms = 0.f;
  HM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  rr.ms = ms;
  rr.truncations = misc[44];
  rr.rand_ok = misc[45];
  rr.rand_fail = misc[46];
  for (int i = 0; i < 6; ++i) rr.bad[i] = misc[47 + i];
  rr.sketch_attempts = misc[53];
  rr.gang = misc[55];
  rr.sketch_cols = misc[54];
  if (lo.record && lo.rec_out) {
    size_t cnt = (size_t)std::min<unsigned long long>(misc[60], (unsigned long long)e.rec_cap);
    lo.rec_out->resize(cnt * 7);
    if (cnt) HM_CUDA(cudaMemcpy(lo.rec_out->data(), D.rec.p, cnt * 7 * sizeof(float), cudaMemcpyDeviceToHost));
  }
  if (e.task_ns) {
    rr.task_ns.resize(D.ntasks);
    HM_CUDA(cudaMemcpy(rr.task_ns.data(), D.tns.p, D.ntasks * sizeof(uint32_t), cudaMemcpyDeviceToHost));
    rr.task_aux.resize(D.ntasks);
    HM_CUDA(cudaMemcpy(rr.task_aux.data(), D.tns.as<uint32_t>() + D.ntasks, D.ntasks * sizeof(uint32_t),
                       cudaMemcpyDeviceToHost));
  }
  rr.status = (int)(misc[2] & 0xffffffffu);
  rr.fail_task = (long long)misc[5] - 1;
  std::memcpy(&rr.flops, &misc[3], sizeof(double));
  std::memcpy(&rr.flops32, &misc[4], sizeof(double));
  std::memcpy(&rr.bytes, &misc[6], sizeof(double));
  return rr;
}

RunResult run_tasks(hmat_ctx* ctx, const Sched& S, double* hbase, int* ranks, double eps, int64_t spin_limit,
                    double* ext0, double* ext1, bool mixed = false) {
  DevSched D;
  if (S.tasks.empty()) return RunResult();
  upload_sched(ctx, S, D);
  return launch_sched(ctx, S, D, hbase, ranks, eps, spin_limit, ext0, ext1, mixed);
}

hmat_ctx* check_ctx(hmat_ctx* ctx) {
  require(ctx != nullptr, "null context");
  HM_CUDA(cudaSetDevice(ctx->device));
  return ctx;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

size_t hmat_last_error(char* buf, size_t size) {
  if (buf && size) {
    size_t n = std::min(size - 1, g_last_error.size());
    std::memcpy(buf, g_last_error.data(), n);
    buf[n] = 0;
  }
  return g_last_error.size();
}

hmat_status hmat_ctx_create(int device, void* cuda_stream, hmat_ctx** out) {
  return guarded([&] {
    require(out != nullptr, "null output");
    int ndev = 0;
    HM_CUDA(cudaGetDeviceCount(&ndev));
    require(device >= 0 && device < ndev, "no such CUDA device");
    HM_CUDA(cudaSetDevice(device));
    auto* c = new hmat_ctx();
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    HM_CUDA(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device));
    HM_CUDA(exec_occupancy(&c->blocks_per_sm));
    if (c->blocks_per_sm < 1) c->blocks_per_sm = 1;
    *out = c;
  });
}

hmat_status hmat_ctx_destroy(hmat_ctx* ctx) {
  return guarded([&] { delete ctx; });
}

hmat_status hmat_clustertree_build(hmat_ctx* ctx, const double* coords, int64_t n, int d, int64_t leaf_size,
                                   hmat_ctree** out) {
  return guarded([&] {
    (void)ctx;
    require(coords && out && n > 0 && (d == 2 || d == 3) && leaf_size >= 1, "cluster tree: bad arguments");
    auto* T = new hmat_ctree();
    T->d = d;
    std::vector<int64_t> idx((size_t)n), tmp((size_t)n);
    for (int64_t i = 0; i < n; ++i) idx[(size_t)i] = i;
    try {
      ct_rec(*T, coords, idx, tmp, 0, n, 0, -1, leaf_size);
    } catch (...) {
      delete T;
      throw;
    }
    T->perm = std::move(idx);
    *out = T;
  });
}

hmat_status hmat_clustertree_perm(const hmat_ctree* ct, int64_t* perm) {
  return guarded([&] {
    require(ct && perm, "null argument");
    std::memcpy(perm, ct->perm.data(), ct->perm.size() * sizeof(int64_t));
  });
}

int64_t hmat_clustertree_size(const hmat_ctree* ct) { return ct ? (int64_t)ct->nodes.size() : 0; }

hmat_status hmat_clustertree_nodes(const hmat_ctree* ct, int64_t* off, int64_t* size, int* level, int* parent,
                                   int* nsons) {
  return guarded([&] {
    require(ct && off && size && level && parent && nsons, "null argument");
    for (size_t i = 0; i < ct->nodes.size(); ++i) {
      off[i] = ct->nodes[i].off;
      size[i] = ct->nodes[i].size;
      level[i] = ct->nodes[i].level;
      parent[i] = ct->nodes[i].parent;
      nsons[i] = ct->nodes[i].nsons;
    }
  });
}

hmat_status hmat_ctree_destroy(hmat_ctree* ct) {
  return guarded([&] { delete ct; });
}

hmat_status hmat_blocktree_build(hmat_ctx* ctx, const hmat_ctree* rows, const hmat_ctree* cols, double eta,
                                 hmat_btree** out) {
  return guarded([&] {
    (void)ctx;
    require(rows && cols && out && rows->d == cols->d && eta > 0, "block tree: bad arguments");
    auto* B = new hmat_btree();
    B->R = rows;
    B->C = cols;
    bt_rec(*B, 0, 0, 0, -1, eta);
    *out = B;
  });
}

int64_t hmat_blocktree_size(const hmat_btree* bt) { return bt ? (int64_t)bt->nodes.size() : 0; }

hmat_status hmat_blocktree_nodes(const hmat_btree* bt, int* t, int* s, int* level, int* parent, int* kind) {
  return guarded([&] {
    require(bt && t && s && level && parent && kind, "null argument");
    for (size_t i = 0; i < bt->nodes.size(); ++i) {
      t[i] = bt->nodes[i].t;
      s[i] = bt->nodes[i].s;
      level[i] = bt->nodes[i].level;
      parent[i] = bt->nodes[i].parent;
      kind[i] = bt->nodes[i].kind;
    }
  });
}

hmat_status hmat_btree_destroy(hmat_btree* bt) {
  return guarded([&] { delete bt; });
}

}  // extern "C"

namespace {
// Host metadata of an H-matrix: storage layout of every leaf, rank slots, and
// which dense leaves hold entries of the sparse matrix.
std::vector<DenseLeafDesc> layout_from_csr(hmat* H, const hmat_btree* bt, int64_t n, const int64_t* rowptr,
                                           const int64_t* colidx, const double* val) {
    H->bt = bt;
    H->n = n;
    size_t nb = bt->nodes.size();
    H->loc.assign(nb, -1);
    H->vloc.assign(nb, -1);
    H->cap.assign(nb, 0);
    H->slot.assign(nb, -1);
    H->zero.assign(nb, 1);
    int64_t off = 0;
    std::vector<DenseLeafDesc> dl;
    for (size_t b = 0; b < nb; ++b) {
      int kind = bt->nodes[b].kind;
      int64_t m = H->rows((int)b), k = H->cols((int)b);
      if (kind == 1) {
        H->loc[b] = off;
        DenseLeafDesc d;
        d.off = off;
        d.roff = H->tc((int)b).off;
        d.coff = H->sc((int)b).off;
        d.rows = (int)m;
        d.cols = (int)k;
        dl.push_back(d);
        off += m * k;
      } else if (kind == 2) {
        int c = (int)std::min<int64_t>(std::min(m, k), H->max_rank);
        H->cap[b] = c;
        H->loc[b] = off;
        off += m * c;
        H->vloc[b] = off;
        off += k * c;
        H->slot[b] = H->nslots++;
      }
    }
    H->store_doubles = off;
    const std::vector<int64_t>& perm = bt->R->perm;
    std::vector<int64_t> iperm((size_t)n);
    for (int64_t i = 0; i < n; ++i) iperm[(size_t)bt->C->perm[(size_t)i]] = i;
    for (size_t b = 0; b < nb; ++b) {
      if (bt->nodes[b].kind != 1) continue;
      const CNodeH& t = H->tc((int)b);
      const CNodeH& s = H->sc((int)b);
      bool any = false;
      for (int64_t i = 0; i < t.size && !any; ++i) {
        int64_t p = perm[(size_t)(t.off + i)];
        for (int64_t e = rowptr[p]; e < rowptr[p + 1]; ++e) {
          int64_t j = iperm[(size_t)colidx[e]];
          if (j >= s.off && j < s.off + s.size && val[e] != 0.0) {
            any = true;
            break;
          }
        }
      }
      H->zero[b] = any ? 0 : 1;
    }
    H->st.n = n;
    H->st.blocks = (int64_t)nb;
    for (size_t b = 0; b < nb; ++b) {
      if (bt->nodes[b].kind == 1) H->st.dense_leaves++;
      if (bt->nodes[b].kind == 2) H->st.lowrank_leaves++;
    }
    return dl;
}

// Checks of the options every factorisation shares: the mode (standard only
// where the call supports it) and the rank rule (the spectral one needs the
// exact FP64 truncations: the mixed form's checks bound Frobenius residuals).
void check_opts(const hmat_opts* opts, bool standard_ok) {
  if (!opts) return;
  require(opts->mode == HMAT_ACCUMULATED || (standard_ok && opts->mode == HMAT_STANDARD),
          standard_ok ? "mode must be HMAT_ACCUMULATED or HMAT_STANDARD" : "this call has the accumulated form only");
  require(opts->rank_rule == HMAT_REL_FRO || opts->rank_rule == HMAT_REL_SPEC, "rank_rule must be REL_FRO or REL_SPEC");
  require(opts->rank_rule == HMAT_REL_FRO || opts->precision == HMAT_FP64,
          "the relative spectral rank rule needs precision HMAT_FP64");
}

// Symbolic H-LU of H into S (ordered by level); returns host seconds.
double schedule_lu(hmat* H, int64_t max_rank, bool mixed, bool standard, Sched& S) {
  auto t0 = std::chrono::steady_clock::now();
  S.reserve_for_blocks(H->bt->nodes.size());
  S.next_slot = H->nslots;
  Sym sym(S, *H->bt->R, *H->bt->C, max_rank);
  sym.mixed = mixed;
  sym.dense_small = mixed;
  sym.add_matrix(H);
  if (standard) {
    sym.lu_std(H, 0);
  } else {
    SAcc root = sym.acc_new(0, 0);
    sym.lu(H, 0, root);
  }
  S.order_by_level();
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}
}  // namespace

extern "C" {

hmat_status hmat_analyze_lu(const hmat_btree* bt, int64_t n, const int64_t* rowptr, const int64_t* colidx,
                            const double* val, const hmat_opts* opts, hmat_stats* out) {
  return guarded([&] {
    require(bt && rowptr && colidx && val && out, "null argument");
    require((int64_t)bt->R->perm.size() == n && (int64_t)bt->C->perm.size() == n, "csr: size does not match the trees");
    hmat H;
    layout_from_csr(&H, bt, n, rowptr, colidx, val);
    int64_t mr = (opts && opts->max_rank > 0) ? std::min<int64_t>(opts->max_rank, H.max_rank) : H.max_rank;
    Sched S;
    check_opts(opts, true);
    double secs = schedule_lu(&H, mr, opts && opts->precision == HMAT_MIXED, opts && opts->mode == HMAT_STANDARD, S);
    hmat_stats s = H.st;
    s.tasks = (int64_t)S.tasks.size();
    s.truncations = 0;  // truncation tasks of the schedule (those whose product is zero skip at run time)
    for (const HTask& t : S.tasks)  // a gang is one truncation
      s.truncations += ((t.type == T_RKADD || t.type == T_ROWMERGE) && (t.pad1 <= 1 || t.pad0 == 0)) ? 1 : 0;
    s.schedule_seconds = secs;
    s.levels = S.levels();
    s.critical_flops = S.critical_flops();
    s.est_flops = S.est_total;
    s.device_bytes = H.store_doubles * 8 + S.ws_top * 8;
    *out = s;
  });
}

hmat_status hmat_create_from_csr(hmat_ctx* ctx, const hmat_btree* bt, int64_t n, const int64_t* rowptr,
                                 const int64_t* colidx, const double* val, hmat** out) {
  return guarded([&] {
    check_ctx(ctx);
    require(bt && rowptr && colidx && val && out, "null argument");
    require((int64_t)bt->R->perm.size() == n && (int64_t)bt->C->perm.size() == n, "csr: size does not match the trees");
    std::unique_ptr<hmat> H(new hmat());
    H->ctx = ctx;
    H->device = ctx->device;
    std::vector<DenseLeafDesc> dl = layout_from_csr(H.get(), bt, n, rowptr, colidx, val);
    int64_t off = H->store_doubles;
    size_t nb = bt->nodes.size();
    cudaStream_t st = ctx->stream;
    H->store.alloc((size_t)std::max<int64_t>(off, 1) * sizeof(double));
    HM_CUDA(cudaMemsetAsync(H->store.p, 0, (size_t)std::max<int64_t>(off, 1) * sizeof(double), st));
    H->ranks.alloc((size_t)std::max(H->nslots, 1) * sizeof(int));
    HM_CUDA(cudaMemsetAsync(H->ranks.p, 0, (size_t)std::max(H->nslots, 1) * sizeof(int), st));
    const std::vector<int64_t>& perm = bt->R->perm;
    std::vector<int64_t> iperm((size_t)n);
    for (int64_t i = 0; i < n; ++i) iperm[(size_t)bt->C->perm[(size_t)i]] = i;
    int64_t nnz = rowptr[n];
    DevBuf drp, dci, dva, dperm, diperm, ddl, dplaced;
    upload(drp, std::vector<int64_t>(rowptr, rowptr + n + 1), st);
    upload(dci, std::vector<int64_t>(colidx, colidx + nnz), st);
    upload(dva, std::vector<double>(val, val + nnz), st);
    upload(dperm, perm, st);
    upload(diperm, iperm, st);
    upload(ddl, dl, st);
    dplaced.alloc(2 * sizeof(unsigned long long));
    HM_CUDA(cudaMemsetAsync(dplaced.p, 0, 2 * sizeof(unsigned long long), st));
    HM_CUDA(launch_csr_scatter(ddl.as<DenseLeafDesc>(), (int)dl.size(), drp.as<int64_t>(), dci.as<int64_t>(),
                               dva.as<double>(), dperm.as<int64_t>(), diperm.as<int64_t>(), H->store.as<double>(),
                               dplaced.as<unsigned long long>(), st));
    unsigned long long placed[2] = {0, 0};
    HM_CUDA(cudaMemcpyAsync(placed, dplaced.p, sizeof(placed), cudaMemcpyDeviceToHost, st));
    HM_CUDA(cudaStreamSynchronize(st));
    require((int64_t)placed[0] == nnz, "csr: entries inside admissible blocks (rank > 0) are not supported");
    if (placed[1])
      throw HmError(HMAT_ERR_NONFINITE, "csr: " + std::to_string(placed[1]) + " non-finite values");
    (void)nb;
    H->st.device_bytes = (int64_t)(H->store.bytes + H->ranks.bytes);
    *out = H.release();
  });
}

hmat_status hmat_destroy(hmat* H) {
  return guarded([&] {
    // the context may already be gone: use the device recorded at creation,
    // and leave no error of this call behind for a later launch check
    if (H) cudaSetDevice(H->device);
    delete H;
    (void)cudaGetLastError();
  });
}

hmat_status hmat_copy_values(hmat_ctx* ctx, hmat* dst, const hmat* src) {
  return guarded([&] {
    check_ctx(ctx);
    require(dst && src && dst->bt == src->bt && dst->store_doubles == src->store_doubles, "copy_values: different trees");
    HM_CUDA(cudaMemcpyAsync(dst->store.p, src->store.p, (size_t)src->store_doubles * sizeof(double),
                            cudaMemcpyDeviceToDevice, ctx->stream));
    HM_CUDA(cudaMemcpyAsync(dst->ranks.p, src->ranks.p, (size_t)src->nslots * sizeof(int), cudaMemcpyDeviceToDevice,
                            ctx->stream));
    dst->zero = src->zero;
  });
}

hmat_status hmat_to_dense(hmat_ctx* ctx, const hmat* H, double* out) {
  return guarded([&] {
    check_ctx(ctx);
    require(H && out, "null argument");
    std::vector<LeafRef> L;
    for (size_t b = 0; b < H->bt->nodes.size(); ++b) {
      int kind = H->bt->nodes[b].kind;
      if (kind == 0) continue;
      LeafRef r;
      std::memset(&r, 0, sizeof(r));
      r.kind = kind;
      r.rows = (int)H->rows((int)b);
      r.cols = (int)H->cols((int)b);
      r.roff = (int)H->tc((int)b).off;
      r.coff = (int)H->sc((int)b).off;
      r.lda = r.rows;
      r.ldb = r.cols;
      r.a = H->loc[b];
      r.b = H->vloc[b];
      r.rank_slot = H->slot[b];
      L.push_back(r);
    }
    DevBuf dl;
    upload(dl, L, ctx->stream);
    HM_CUDA(launch_to_dense(dl.as<LeafRef>(), (int)L.size(), H->store.as<double>(), H->ranks.as<int>(), out, H->n,
                            ctx->stream));
    HM_CUDA(cudaStreamSynchronize(ctx->stream));
  });
}

hmat_status hmat_addeval(hmat_ctx* ctx, const hmat* H, double alpha, int trans, int64_t ncol, const double* X,
                         double* Y) {
  return guarded([&] {
    check_ctx(ctx);
    require(H && X && Y && ncol >= 0, "addeval: bad arguments");
    if (ncol == 0) return;
    Sched S;
    S.next_slot = H->nslots;
    Sym sym(S, *H->bt->R, *H->bt->C, H->max_rank);
    sym.add_matrix(H);
    int xobj = S.new_obj(), yobj_base = (int)S.objs.size();
    // Output rows are split by the clusters of the shallowest level at which
    // leaves start, so that independent CTAs write disjoint rows.
    const hmat_btree& B = *H->bt;
    int lmin = 1 << 30;
    for (const BNodeH& nd : B.nodes)
      if (nd.kind != 0) lmin = std::min(lmin, trans ? B.C->nodes[(size_t)nd.s].level : B.R->nodes[(size_t)nd.t].level);
    const hmat_ctree& OT = trans ? *B.C : *B.R;
    std::vector<int> groups;
    for (size_t c = 0; c < OT.nodes.size(); ++c)
      if (OT.nodes[c].level == lmin || (OT.nodes[c].level < lmin && OT.nodes[c].nsons == 0)) groups.push_back((int)c);
    std::vector<std::vector<LeafRef>> per((size_t)OT.nodes.size());
    std::vector<std::vector<int>> reads((size_t)OT.nodes.size());
    std::vector<int> owner(OT.nodes.size(), -1);
    for (int g : groups) {
      // every descendant maps to its group
      std::vector<int> st{g};
      while (!st.empty()) {
        int c = st.back();
        st.pop_back();
        owner[(size_t)c] = g;
        for (int k = 0; k < OT.nodes[(size_t)c].nsons; ++k) st.push_back(OT.nodes[(size_t)c].son[k]);
      }
    }
    std::vector<LeafRef> all;
    std::vector<int> objs;
    sym.collect(H, 0, 0, 0, true, all, objs);
    for (size_t i = 0; i < all.size(); ++i) {
      // find the leaf's output cluster by its offset
      const LeafRef& L = all[i];
      int64_t o = trans ? L.coff : L.roff;
      int g = -1;
      for (int c : groups)
        if (OT.nodes[(size_t)c].off <= o && o < OT.nodes[(size_t)c].off + OT.nodes[(size_t)c].size) g = c;
      per[(size_t)g].push_back(L);
      reads[(size_t)g].push_back(objs[i]);
    }
    (void)owner;
    for (int g : groups) {
      if (per[(size_t)g].empty()) continue;
      HTask t = blank(T_HMV);
      t.flags = trans ? F_TRANS : 0;
      t.m = (int)OT.nodes[(size_t)g].size;
      t.alpha = alpha;
      t.b = tag_ext(0, 0);
      t.ldb = (int)H->n;
      t.c = tag_ext(1, 0);
      t.ldc = (int)H->n;
      t.wa = (int)ncol;
      t.list_begin = (int)S.leaves.size();
      t.list_len = (int)per[(size_t)g].size();
      S.leaves.insert(S.leaves.end(), per[(size_t)g].begin(), per[(size_t)g].end());
      std::vector<int> rd = reads[(size_t)g];
      rd.push_back(xobj);
      int yo = S.new_obj();
      S.emit(t, rd, {yo});
    }
    (void)yobj_base;
    RunResult rr = run_tasks(ctx, S, H->store.as<double>(), H->ranks.as<int>(), 0.0, 0, (double*)X, Y);
    if (rr.status) throw HmError(rr.status, "addeval: device status");
  });
}

}  // extern "C"

// A factorisation schedule kept for reuse: it depends only on the block
// trees, the storage layout, the initial zero pattern of the leaves, max_rank
// and the precision, never on the values.
struct SchedCache {
  std::vector<const hmat*> mats;
  std::vector<const hmat_btree*> trees;
  std::vector<uint64_t> zero_hash;
  std::vector<std::vector<char>> zero_after;
  int64_t mr = 0;
  bool mixed = false;
  int mode = HMAT_ACCUMULATED;
  double* base = nullptr;
  Sched S;
  DevSched D;
};

namespace {
uint64_t hash_flags(const std::vector<char>& v) {
  uint64_t h = 1469598103934665603ull;  // FNV-1a
  for (char c : v) h = (h ^ (uint64_t)(unsigned char)c) * 1099511628211ull;
  return h ^ v.size();
}

// H-LU of count independent H-matrices in one schedule and one persistent
// launch.  Storage locations are offsets from the lowest storage pointer of
// the batch; each instance's leaf rank slots get their own range.
void lu_batch(hmat_ctx* ctx, hmat* const* Hs, int count, const hmat_opts* opts) {
  check_ctx(ctx);
  check_opts(opts, true);
  require(Hs != nullptr && count >= 1, "no H-matrices");
  for (int i = 0; i < count; ++i) require(Hs[i] != nullptr && Hs[i]->ctx == ctx, "null H-matrix or other context");
  double eps = opts ? opts->eps : 0.0;
  int64_t spin = opts ? opts->spin_limit : 0;
  require(eps >= 0.0, "eps must be >= 0");
  bool mixed = opts && opts->precision == HMAT_MIXED;
  auto t0 = std::chrono::steady_clock::now();
  double* base = Hs[0]->store.as<double>();
  for (int i = 1; i < count; ++i) base = std::min(base, Hs[i]->store.as<double>());
  std::vector<int> slotbase((size_t)count, 0);
  int nslots = 0;
  for (int i = 0; i < count; ++i) {
    slotbase[(size_t)i] = nslots;
    nslots += Hs[i]->nslots;
  }
  int64_t mr0 = (opts && opts->max_rank > 0) ? opts->max_rank : DEFAULT_MAX_RANK;
  std::vector<uint64_t> zh((size_t)count);
  for (int i = 0; i < count; ++i) zh[(size_t)i] = hash_flags(Hs[i]->zero);
  bool reuse = opts && opts->reuse_schedule;
  SchedCache* C = Hs[0]->cache.get();
  bool standard = opts && opts->mode == HMAT_STANDARD;
  bool hit = reuse && C && C->mixed == mixed && C->mode == (standard ? HMAT_STANDARD : HMAT_ACCUMULATED) &&
             C->mr == mr0 && C->base == base && (int)C->mats.size() == count &&
             C->zero_hash == zh;
  for (int i = 0; hit && i < count; ++i) hit = C->mats[(size_t)i] == Hs[i] && C->trees[(size_t)i] == Hs[i]->bt;
  std::shared_ptr<SchedCache> fresh;
  if (!hit) {
    fresh = std::make_shared<SchedCache>();
    C = fresh.get();
  }
  Sched& S = C->S;
  if (!hit) {
  size_t nblocks = 0;
  for (int i = 0; i < count; ++i) nblocks += Hs[i]->bt->nodes.size();
  S.reserve_for_blocks(nblocks);
  S.next_slot = nslots;
  for (int i = 0; i < count; ++i) {
    hmat* H = Hs[i];
    int64_t mr = std::min<int64_t>(mr0, H->max_rank);
    S.set_pool(i);
    Sym sym(S, *H->bt->R, *H->bt->C, mr);
    sym.mixed = mixed;
    sym.dense_small = mixed;
    sym.add_matrix(H, (int64_t)(H->store.as<double>() - base), slotbase[(size_t)i]);
    if (standard) {
      sym.lu_std(H, 0);
    } else {
      SAcc root = sym.acc_new(0, 0);
      sym.lu(H, 0, root);
    }
  }
  S.order_by_level();
  upload_sched(ctx, S, C->D);
  for (int i = 0; i < count; ++i) {
    C->mats.push_back(Hs[i]);
    C->trees.push_back(Hs[i]->bt);
    C->zero_after.push_back(Hs[i]->zero);
  }
  C->zero_hash = zh;
  C->mr = mr0;
  C->mixed = mixed;
  C->mode = standard ? HMAT_STANDARD : HMAT_ACCUMULATED;
  C->base = base;
  if (reuse) Hs[0]->cache = fresh;
  } else {
    for (int i = 0; i < count; ++i) Hs[i]->zero = C->zero_after[(size_t)i];
  }
  double sched_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  DevBuf allranks((size_t)std::max(S.next_slot, 1) * sizeof(int));
  for (int i = 0; i < count; ++i)
    HM_CUDA(cudaMemcpyAsync(allranks.as<int>() + slotbase[(size_t)i], Hs[i]->ranks.p, (size_t)Hs[i]->nslots * sizeof(int),
                            cudaMemcpyDeviceToDevice, ctx->stream));
  LaunchOpts lo;
  lo.mlp = opts ? hm_internal::mlp_weights(opts->predictor) : nullptr;
  lo.record = opts && opts->record_training;
  lo.rec_out = &Hs[0]->train;
  lo.seed = opts ? opts->seed : 0;
  lo.rank_rule = opts ? opts->rank_rule : 0;
  RunResult rr = launch_sched(ctx, S, C->D, base, allranks.as<int>(), eps, spin, nullptr, nullptr, mixed, lo);
  for (int i = 0; i < count; ++i)
    HM_CUDA(cudaMemcpyAsync(Hs[i]->ranks.p, allranks.as<int>() + slotbase[(size_t)i], (size_t)Hs[i]->nslots * sizeof(int),
                            cudaMemcpyDeviceToDevice, ctx->stream));
  HM_CUDA(cudaStreamSynchronize(ctx->stream));
  if (rr.bad[0]) {
    double sc;
    std::memcpy(&sc, &rr.bad[5], sizeof(sc));
    std::fprintf(stderr, "hmat_lu: non-finite randomised result redone exactly (path %llu, m %llu, n %llu, l %llu, k %llu, scale %g)\n",
                 rr.bad[0], rr.bad[1], rr.bad[2], rr.bad[3], rr.bad[4], sc);
  }
  for (int i = 0; i < count; ++i) {
    hmat_stats& st = Hs[i]->st;  // the batch's totals, on every instance
    st.tasks = (int64_t)S.tasks.size();
    st.truncations = (int64_t)rr.truncations;
    st.flops = rr.flops;
    st.flops32 = rr.flops32;
    st.bytes = rr.bytes;
    st.gang_truncations = (int64_t)rr.gang;
    st.rand_truncations = (int64_t)rr.rand_ok;
    st.rand_fallbacks = (int64_t)rr.rand_fail;
    st.sketch_attempts = (int64_t)rr.sketch_attempts;
    st.sketch_columns = (int64_t)rr.sketch_cols;
    st.training_pairs = (int64_t)(Hs[0]->train.size() / 7);
    if (!rr.task_ns.empty()) critical_path(S, rr.task_ns, rr.task_aux, st);
    for (int k = 0; k < 16; ++k) {
      st.type_seconds[k] = rr.type_ns[k] * 1e-9;
      st.type_count[k] = (int64_t)rr.type_cnt[k];
    }
    st.wait_seconds = rr.wait_ns * 1e-9;
    st.factor_seconds = rr.ms * 1e-3;
    st.schedule_seconds = sched_s;
    st.schedule_reused = hit ? 1 : 0;
    st.status = rr.status;
    st.levels = S.levels();
    st.critical_flops = S.critical_flops();
    st.est_flops = S.est_total;
    st.device_bytes = (int64_t)(Hs[i]->store.bytes + Hs[i]->ranks.bytes) + S.ws_top * 8;
  }
  if (rr.status)
    throw HmError(rr.status, "hmat_lu: device status " + std::to_string(rr.status) +
                                 describe_failure(S, rr.fail_task, Hs, count, base));
}

// In-place H-Cholesky with accumulated updates: one schedule, one launch.
void chol_run(hmat_ctx* ctx, hmat* G, const hmat_opts* opts) {
  check_ctx(ctx);
  check_opts(opts, false);
  require(G && G->ctx == ctx, "null H-matrix or other context");
  double eps = opts ? opts->eps : 0.0;
  require(eps >= 0.0, "eps must be >= 0");
  int64_t spin = opts ? opts->spin_limit : 0;
  bool mixed = opts && opts->precision == HMAT_MIXED;
  auto t0 = std::chrono::steady_clock::now();
  int64_t mr = (opts && opts->max_rank > 0) ? opts->max_rank : DEFAULT_MAX_RANK;
  mr = std::min<int64_t>(mr, G->max_rank);
  Sched S;
  DevSched D;
  S.next_slot = G->nslots;
  S.set_pool(0);
  Sym sym(S, *G->bt->R, *G->bt->C, mr);
  sym.mixed = mixed;
  sym.dense_small = mixed;
  sym.add_matrix(G);
  SAcc root = sym.acc_new(0, 0);
  sym.chol(G, 0, root);
  S.order_by_level();
  upload_sched(ctx, S, D);
  double sched_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  DevBuf allranks((size_t)std::max(S.next_slot, 1) * sizeof(int));
  HM_CUDA(cudaMemcpyAsync(allranks.as<int>(), G->ranks.p, (size_t)G->nslots * sizeof(int), cudaMemcpyDeviceToDevice,
                          ctx->stream));
  LaunchOpts lo;
  lo.mlp = opts ? hm_internal::mlp_weights(opts->predictor) : nullptr;
  lo.record = opts && opts->record_training;
  lo.rec_out = &G->train;
  lo.seed = opts ? opts->seed : 0;
  lo.rank_rule = opts ? opts->rank_rule : 0;
  RunResult rr = launch_sched(ctx, S, D, G->store.as<double>(), allranks.as<int>(), eps, spin, nullptr, nullptr,
                              mixed, lo);
  HM_CUDA(cudaMemcpyAsync(G->ranks.p, allranks.as<int>(), (size_t)G->nslots * sizeof(int), cudaMemcpyDeviceToDevice,
                          ctx->stream));
  HM_CUDA(cudaStreamSynchronize(ctx->stream));
  G->cache.reset();
  hmat_stats& st = G->st;
  st.tasks = (int64_t)S.tasks.size();
  st.truncations = (int64_t)rr.truncations;
  st.flops = rr.flops;
  st.flops32 = rr.flops32;
  st.bytes = rr.bytes;
  st.gang_truncations = (int64_t)rr.gang;
  st.rand_truncations = (int64_t)rr.rand_ok;
  st.rand_fallbacks = (int64_t)rr.rand_fail;
  st.sketch_attempts = (int64_t)rr.sketch_attempts;
  st.sketch_columns = (int64_t)rr.sketch_cols;
  if (!rr.task_ns.empty()) critical_path(S, rr.task_ns, rr.task_aux, st);
  for (int k = 0; k < 16; ++k) {
    st.type_seconds[k] = rr.type_ns[k] * 1e-9;
    st.type_count[k] = (int64_t)rr.type_cnt[k];
  }
  st.wait_seconds = rr.wait_ns * 1e-9;
  st.factor_seconds = rr.ms * 1e-3;
  st.schedule_seconds = sched_s;
  st.schedule_reused = 0;
  st.status = rr.status;
  st.levels = S.levels();
  st.critical_flops = S.critical_flops();
  st.est_flops = S.est_total;
  st.device_bytes = (int64_t)(G->store.bytes + G->ranks.bytes) + S.ws_top * 8;
  if (rr.status) {
    hmat* Gs[1] = {G};
    throw HmError(rr.status, "hmat_cholesky: device status " + std::to_string(rr.status) +
                                 describe_failure(S, rr.fail_task, Gs, 1, G->store.as<double>()));
  }
}

// In-place H-inversion with accumulated updates (Fig. invert): the auxiliary
// H-matrix for H_12, H_21 lives for the call; one schedule, one launch.
void invert_run(hmat_ctx* ctx, hmat* G, const hmat_opts* opts) {
  check_ctx(ctx);
  check_opts(opts, false);
  require(G && G->ctx == ctx, "null H-matrix or other context");
  double eps = opts ? opts->eps : 0.0;
  require(eps >= 0.0, "eps must be >= 0");
  int64_t spin = opts ? opts->spin_limit : 0;
  bool mixed = opts && opts->precision == HMAT_MIXED;
  auto t0 = std::chrono::steady_clock::now();
  // auxiliary H-matrix: the layout of G, all leaves zero
  std::unique_ptr<hmat> H(new hmat());
  H->ctx = ctx;
  H->device = ctx->device;
  {
    std::vector<int64_t> rp((size_t)G->n + 1, 0);
    int64_t dummy_i = 0;
    double dummy_v = 0.0;
    layout_from_csr(H.get(), G->bt, G->n, rp.data(), &dummy_i, &dummy_v);
    H->store.alloc((size_t)std::max<int64_t>(H->store_doubles, 1) * sizeof(double));
    HM_CUDA(cudaMemsetAsync(H->store.p, 0, (size_t)std::max<int64_t>(H->store_doubles, 1) * sizeof(double),
                            ctx->stream));
    H->ranks.alloc((size_t)std::max(H->nslots, 1) * sizeof(int));
    HM_CUDA(cudaMemsetAsync(H->ranks.p, 0, (size_t)std::max(H->nslots, 1) * sizeof(int), ctx->stream));
  }
  hmat* M[2] = {G, H.get()};
  double* base = std::min(G->store.as<double>(), H->store.as<double>());
  int slotbase[2] = {0, G->nslots};
  int64_t mr = (opts && opts->max_rank > 0) ? opts->max_rank : DEFAULT_MAX_RANK;
  mr = std::min<int64_t>(mr, G->max_rank);
  Sched S;
  DevSched D;
  S.next_slot = G->nslots + H->nslots;
  S.set_pool(0);
  Sym sym(S, *G->bt->R, *G->bt->C, mr);
  sym.mixed = mixed;
  // dense small accumulators pay in the LU only: in the multiplication and the
  // inversion (32^3) they cost 3.6x and 5.1x the time of low-rank ones
  sym.dense_small = false;
  for (int i = 0; i < 2; ++i) sym.add_matrix(M[i], (int64_t)(M[i]->store.as<double>() - base), slotbase[i]);
  SAcc root = sym.acc_new(0, 0);
  sym.invert(G, H.get(), 0, root);
  S.order_by_level();
  upload_sched(ctx, S, D);
  double sched_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  DevBuf allranks((size_t)std::max(S.next_slot, 1) * sizeof(int));
  for (int i = 0; i < 2; ++i)
    HM_CUDA(cudaMemcpyAsync(allranks.as<int>() + slotbase[i], M[i]->ranks.p, (size_t)M[i]->nslots * sizeof(int),
                            cudaMemcpyDeviceToDevice, ctx->stream));
  LaunchOpts lo;
  lo.mlp = opts ? hm_internal::mlp_weights(opts->predictor) : nullptr;
  lo.record = opts && opts->record_training;
  lo.rec_out = &G->train;
  lo.seed = opts ? opts->seed : 0;
  lo.rank_rule = opts ? opts->rank_rule : 0;
  RunResult rr = launch_sched(ctx, S, D, base, allranks.as<int>(), eps, spin, nullptr, nullptr, mixed, lo);
  HM_CUDA(cudaMemcpyAsync(G->ranks.p, allranks.as<int>(), (size_t)G->nslots * sizeof(int), cudaMemcpyDeviceToDevice,
                          ctx->stream));
  HM_CUDA(cudaStreamSynchronize(ctx->stream));
  G->cache.reset();  // a kept LU schedule no longer describes G's zero pattern
  hmat_stats& st = G->st;
  st.tasks = (int64_t)S.tasks.size();
  st.truncations = (int64_t)rr.truncations;
  st.flops = rr.flops;
  st.flops32 = rr.flops32;
  st.bytes = rr.bytes;
  st.gang_truncations = (int64_t)rr.gang;
  st.rand_truncations = (int64_t)rr.rand_ok;
  st.rand_fallbacks = (int64_t)rr.rand_fail;
  st.sketch_attempts = (int64_t)rr.sketch_attempts;
  st.sketch_columns = (int64_t)rr.sketch_cols;
  st.training_pairs = (int64_t)(G->train.size() / 7);
  if (!rr.task_ns.empty()) critical_path(S, rr.task_ns, rr.task_aux, st);
  for (int k = 0; k < 16; ++k) {
    st.type_seconds[k] = rr.type_ns[k] * 1e-9;
    st.type_count[k] = (int64_t)rr.type_cnt[k];
  }
  st.wait_seconds = rr.wait_ns * 1e-9;
  st.factor_seconds = rr.ms * 1e-3;
  st.schedule_seconds = sched_s;
  st.schedule_reused = 0;
  st.status = rr.status;
  st.levels = S.levels();
  st.critical_flops = S.critical_flops();
  st.est_flops = S.est_total;
  st.device_bytes = (int64_t)(G->store.bytes + G->ranks.bytes + H->store.bytes) + S.ws_top * 8;
  if (rr.status) throw HmError(rr.status, "hmat_invert: device status " + std::to_string(rr.status));
}

// Z <- blocktrunc(Z + alpha X Y) in the accumulated form: one addproduct at
// the root pair, one flush into Z, one launch.
void addmul_run(hmat_ctx* ctx, double alpha, const hmat* X, const hmat* Y, hmat* Z, const hmat_opts* opts) {
  check_ctx(ctx);
  check_opts(opts, true);
  require(X && Y && Z, "null H-matrix");
  require(X->ctx == ctx && Y->ctx == ctx && Z->ctx == ctx, "H-matrix of another context");
  require(Z != X && Z != Y, "addmul: Z must not be X or Y");
  const hmat_ctree* T = Z->bt->R;
  require(Z->bt->C == T && X->bt->R == T && X->bt->C == T && Y->bt->R == T && Y->bt->C == T,
          "addmul: X, Y and Z must be built on one cluster tree");
  double eps = opts ? opts->eps : 0.0;
  require(eps >= 0.0, "eps must be >= 0");
  int64_t spin = opts ? opts->spin_limit : 0;
  bool mixed = opts && opts->precision == HMAT_MIXED;
  auto t0 = std::chrono::steady_clock::now();
  const hmat* M[3] = {X, Y, Z};
  double* base = X->store.as<double>();
  for (int i = 1; i < 3; ++i) base = std::min(base, M[i]->store.as<double>());
  int slotbase[3];
  int nslots = 0;
  for (int i = 0; i < 3; ++i) {
    slotbase[i] = nslots;
    nslots += M[i]->nslots;
  }
  int64_t mr = (opts && opts->max_rank > 0) ? opts->max_rank : DEFAULT_MAX_RANK;
  mr = std::min<int64_t>(mr, Z->max_rank);
  Sched S;
  DevSched D;
  S.next_slot = nslots;
  S.set_pool(0);
  Sym sym(S, *T, *T, mr);
  sym.mixed = mixed;
  // dense small accumulators pay in the LU only: in the multiplication and the
  // inversion (32^3) they cost 3.6x and 5.1x the time of low-rank ones
  sym.dense_small = false;
  for (int i = 0; i < 3; ++i) sym.add_matrix(M[i], (int64_t)(M[i]->store.as<double>() - base), slotbase[i]);
  STarget z;
  z.M = Z;
  z.b = 0;
  z.t = 0;
  z.r = 0;
  if (opts && opts->mode == HMAT_STANDARD) {
    sym.mult_std(alpha, X, 0, Y, 0, z);
  } else {
    SAcc root = sym.acc_new(0, 0);
    sym.addproduct(alpha, X, 0, Y, 0, root);
    sym.flush(root, z);
  }
  S.order_by_level();
  upload_sched(ctx, S, D);
  double sched_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  DevBuf allranks((size_t)std::max(S.next_slot, 1) * sizeof(int));
  for (int i = 0; i < 3; ++i)
    HM_CUDA(cudaMemcpyAsync(allranks.as<int>() + slotbase[i], M[i]->ranks.p, (size_t)M[i]->nslots * sizeof(int),
                            cudaMemcpyDeviceToDevice, ctx->stream));
  LaunchOpts lo;
  lo.mlp = opts ? hm_internal::mlp_weights(opts->predictor) : nullptr;
  lo.record = opts && opts->record_training;
  lo.rec_out = &Z->train;
  lo.seed = opts ? opts->seed : 0;
  lo.rank_rule = opts ? opts->rank_rule : 0;
  RunResult rr = launch_sched(ctx, S, D, base, allranks.as<int>(), eps, spin, nullptr, nullptr, mixed, lo);
  HM_CUDA(cudaMemcpyAsync(Z->ranks.p, allranks.as<int>() + slotbase[2], (size_t)Z->nslots * sizeof(int),
                          cudaMemcpyDeviceToDevice, ctx->stream));
  HM_CUDA(cudaStreamSynchronize(ctx->stream));
  hmat_stats& st = Z->st;
  st.tasks = (int64_t)S.tasks.size();
  st.truncations = (int64_t)rr.truncations;
  st.flops = rr.flops;
  st.flops32 = rr.flops32;
  st.bytes = rr.bytes;
  st.gang_truncations = (int64_t)rr.gang;
  st.rand_truncations = (int64_t)rr.rand_ok;
  st.rand_fallbacks = (int64_t)rr.rand_fail;
  st.sketch_attempts = (int64_t)rr.sketch_attempts;
  st.sketch_columns = (int64_t)rr.sketch_cols;
  st.training_pairs = (int64_t)(Z->train.size() / 7);
  if (!rr.task_ns.empty()) critical_path(S, rr.task_ns, rr.task_aux, st);
  for (int k = 0; k < 16; ++k) {
    st.type_seconds[k] = rr.type_ns[k] * 1e-9;
    st.type_count[k] = (int64_t)rr.type_cnt[k];
  }
  st.wait_seconds = rr.wait_ns * 1e-9;
  st.factor_seconds = rr.ms * 1e-3;
  st.schedule_seconds = sched_s;
  st.schedule_reused = 0;
  st.status = rr.status;
  st.levels = S.levels();
  st.critical_flops = S.critical_flops();
  st.est_flops = S.est_total;
  st.device_bytes = (int64_t)(Z->store.bytes + Z->ranks.bytes) + S.ws_top * 8;
  if (rr.status) throw HmError(rr.status, "hmat_addmul: device status " + std::to_string(rr.status));
}
}  // namespace

extern "C" {

hmat_status hmat_lu(hmat_ctx* ctx, hmat* H, const hmat_opts* opts) {
  return guarded([&] { lu_batch(ctx, &H, 1, opts); });
}

hmat_status hmat_lu_batched(hmat_ctx* ctx, hmat** G, int count, const hmat_opts* opts) {
  return guarded([&] { lu_batch(ctx, G, count, opts); });
}

hmat_status hmat_addmul(hmat_ctx* ctx, double alpha, const hmat* X, const hmat* Y, hmat* Z, const hmat_opts* opts) {
  return guarded([&] { addmul_run(ctx, alpha, X, Y, Z, opts); });
}

hmat_status hmat_invert(hmat_ctx* ctx, hmat* G, const hmat_opts* opts) {
  return guarded([&] { invert_run(ctx, G, opts); });
}

hmat_status hmat_cholesky(hmat_ctx* ctx, hmat* G, const hmat_opts* opts) {
  return guarded([&] { chol_run(ctx, G, opts); });
}

hmat_status hmat_solve(hmat_ctx* ctx, const hmat* LU, int trans, int64_t nrhs, double* B, int64_t ldb) {
  return guarded([&] {
    check_ctx(ctx);
    require(LU && B && nrhs >= 0 && ldb >= LU->n, "solve: bad arguments");
    if (nrhs == 0) return;
    Sched S;
    S.next_slot = LU->nslots;
    Sym sym(S, *LU->bt->R, *LU->bt->C, LU->max_rank);
    sym.add_matrix(LU);
    int bobj = S.new_obj();
    int64_t x = tag_ext(0, 0);
    if (!trans) {
      sym.hsolve(LU, 0, TRSM_L, x, (int)ldb, bobj, (int)nrhs);
      sym.hsolve(LU, 0, TRSM_U, x, (int)ldb, bobj, (int)nrhs);
    } else {
      sym.hsolve(LU, 0, TRSM_UT, x, (int)ldb, bobj, (int)nrhs);
      sym.hsolve(LU, 0, TRSM_LT, x, (int)ldb, bobj, (int)nrhs);
    }
    RunResult rr = run_tasks(ctx, S, LU->store.as<double>(), LU->ranks.as<int>(), 0.0, 0, B, nullptr);
    if (rr.status) throw HmError(rr.status, "solve: device status");
  });
}

// Extra scratch (doubles) of one problem of trunc_lowrank_batched in the
// mixed form: the explicit FP32 path (M, sketch panels, signs) or the
// factored one (FP32 copies, Mhat, Q_B, panels; tau, R diagonal, core).
static int64_t mixed_ws(int64_t m, int64_t n, int64_t l) {
  int64_t expl = (m * n + 2 * (m + n) * RMAX + n) / 2 + 64;
  int64_t fact = (2 * (m + n) * l + 2 * (m + l) * RMAX + l + 3) / 2 + 2 * l + l * RMAX + 64;
  return std::max(expl, fact);
}

hmat_status trunc_lowrank_batched(hmat_ctx* ctx, int64_t count, const int64_t* m, const int64_t* n, const int64_t* k,
                                  double* const* U, double* const* V, double eps, int64_t* k_new, int precision,
                                  int64_t* randomised) {
  return guarded([&] {
    check_ctx(ctx);
    require(count >= 0 && (count == 0 || (m && n && k && U && V && k_new)), "trunc_lowrank_batched: bad arguments");
    if (count == 0) return;
    int64_t total = 0;
    std::vector<TruncProblem> P((size_t)count);
    for (int64_t i = 0; i < count; ++i) {
      require(m[i] >= 0 && n[i] >= 0 && k[i] >= 0 && k[i] <= HM_LMAX_HOST, "trunc_lowrank: k must be <= 256");
      total += (2 * m[i] + n[i]) * k[i] + 2 * k[i] * k[i] + 64 + (precision == HMAT_MIXED ? mixed_ws(m[i], n[i], k[i]) : 0);
    }
    DevBuf ws((size_t)total * sizeof(double));
    int64_t off = 0;
    for (int64_t i = 0; i < count; ++i) {
      TruncProblem& p = P[(size_t)i];
      p.m = (int)m[i];
      p.n = (int)n[i];
      p.k = (int)k[i];
      p.ldu = (int)std::max<int64_t>(m[i], 1);
      p.ldv = (int)std::max<int64_t>(n[i], 1);
      p.U = U[i];
      p.V = V[i];
      p.ws = ws.as<double>() + off;
      p.k_new = k_new + i;
      off += (2 * m[i] + n[i]) * k[i] + 2 * k[i] * k[i] + 64 + (precision == HMAT_MIXED ? mixed_ws(m[i], n[i], k[i]) : 0);
    }
    DevBuf dp, dst(2 * sizeof(int));
    upload(dp, P, ctx->stream);
    HM_CUDA(cudaMemsetAsync(dst.p, 0, 2 * sizeof(int), ctx->stream));
    HM_CUDA(launch_trunc_batched(dp.as<TruncProblem>(), (int)count, eps, dst.as<int>(), precision == HMAT_MIXED ? 1 : 0,
                                 ctx->stream));
    int status[2] = {0, 0};
    HM_CUDA(cudaMemcpyAsync(status, dst.p, sizeof(status), cudaMemcpyDeviceToHost, ctx->stream));
    HM_CUDA(cudaStreamSynchronize(ctx->stream));
    if (randomised) *randomised = status[1];
    if (status[0]) throw HmError(status[0], "trunc_lowrank: device status");
  });
}

hmat_status hmat_pcg(hmat_ctx* ctx, const hmat* LU, int64_t n, const int64_t* rowptr, const int64_t* colidx,
                     const double* val, int64_t nrhs, const double* B, double* X, double rtol, int64_t maxit,
                     int64_t* iters, double* relres) {
  return guarded([&] {
    check_ctx(ctx);
    require(LU && rowptr && colidx && val && B && X && iters && relres && nrhs >= 0 && maxit >= 0,
            "pcg: bad arguments");
    require(n == LU->n, "pcg: size does not match the factors");
    require(rtol >= 0.0, "pcg: rtol must be >= 0");
    if (nrhs == 0 || n == 0) return;
    cudaStream_t st = ctx->stream;
    // the CSR in the permuted ordering of the factors
    const std::vector<int64_t>& perm = LU->bt->R->perm;
    std::vector<int64_t> iperm((size_t)n);
    for (int64_t i = 0; i < n; ++i) iperm[(size_t)perm[(size_t)i]] = i;
    std::vector<int64_t> prp((size_t)n + 1, 0), pci;
    std::vector<double> pva;
    pci.reserve((size_t)rowptr[n]);
    pva.reserve((size_t)rowptr[n]);
    for (int64_t i = 0; i < n; ++i) {
      int64_t r = perm[(size_t)i];
      for (int64_t e = rowptr[r]; e < rowptr[r + 1]; ++e) {
        require(colidx[e] >= 0 && colidx[e] < n, "pcg: column index out of range");
        require(std::isfinite(val[e]), "pcg: non-finite matrix value");
        pci.push_back(iperm[(size_t)colidx[e]]);
        pva.push_back(val[e]);
      }
      prp[(size_t)i + 1] = (int64_t)pci.size();
    }
    DevBuf drp, dci, dva, dperm;
    upload(drp, prp, st);
    upload(dci, pci, st);
    upload(dva, pva, st);
    upload(dperm, perm, st);
    size_t blk = (size_t)n * nrhs * sizeof(double);
    DevBuf Bp(blk), Xp(blk), R(blk), Z(blk), P(blk), Q(blk), dd(3 * nrhs * sizeof(double));
    double* dscal = dd.as<double>();
    // the solve with the factors as a schedule built once (L then U, Fig. addeval leaves)
    Sched S;
    S.next_slot = LU->nslots;
    Sym sym(S, *LU->bt->R, *LU->bt->C, LU->max_rank);
    sym.add_matrix(LU);
    int zobj = S.new_obj();
    int64_t zx = tag_ext(0, 0);
    sym.hsolve(LU, 0, TRSM_L, zx, (int)n, zobj, (int)nrhs);
    sym.hsolve(LU, 0, TRSM_U, zx, (int)n, zobj, (int)nrhs);
    DevSched D;
    upload_sched(ctx, S, D);
    auto precond = [&]() {  // Z <- (LU)^{-1} R
      HM_CUDA(cudaMemcpyAsync(Z.p, R.p, blk, cudaMemcpyDeviceToDevice, st));
      RunResult rr = launch_sched(ctx, S, D, LU->store.as<double>(), LU->ranks.as<int>(), 0.0, 0, Z.as<double>(),
                                  nullptr, false);
      if (rr.status) throw HmError(rr.status, "pcg: device status of the preconditioner solve");
    };
    std::vector<double> h(3 * (size_t)nrhs);
    auto dots = [&](const DevBuf& a, const DevBuf& b, int slot) {  // into h[slot * nrhs ..]
      HM_CUDA(launch_col_dots(n, nrhs, a.as<double>(), b.as<double>(), dscal + slot * nrhs, st));
    };
    auto fetch = [&]() {
      HM_CUDA(cudaMemcpyAsync(h.data(), dscal, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
      HM_CUDA(cudaStreamSynchronize(st));
    };
    HM_CUDA(launch_permute(B, Bp.as<double>(), dperm.as<int64_t>(), n, nrhs, true, st));
    HM_CUDA(cudaMemsetAsync(Xp.p, 0, blk, st));
    HM_CUDA(cudaMemcpyAsync(R.p, Bp.p, blk, cudaMemcpyDeviceToDevice, st));
    precond();
    HM_CUDA(cudaMemcpyAsync(P.p, Z.p, blk, cudaMemcpyDeviceToDevice, st));
    dots(R, Z, 0);
    dots(Bp, Bp, 1);
    dots(R, R, 2);
    fetch();
    std::vector<double> rz(h.begin(), h.begin() + nrhs), nb((size_t)nrhs), rr2(h.begin() + 2 * nrhs, h.end());
    for (int64_t c = 0; c < nrhs; ++c) {
      nb[(size_t)c] = std::sqrt(h[(size_t)(nrhs + c)]);
      iters[c] = 0;
    }
    std::vector<double> coef((size_t)nrhs);
    for (int64_t it = 0; it < maxit; ++it) {
      std::vector<char> active((size_t)nrhs);
      bool any = false;
      for (int64_t c = 0; c < nrhs; ++c) {
        active[(size_t)c] = std::sqrt(rr2[(size_t)c]) > rtol * nb[(size_t)c];
        any = any || active[(size_t)c];
      }
      if (!any) break;
      HM_CUDA(launch_csr_spmv(n, drp.as<int64_t>(), dci.as<int64_t>(), dva.as<double>(), P.as<double>(),
                              Q.as<double>(), nrhs, st));
      dots(P, Q, 0);
      fetch();
      for (int64_t c = 0; c < nrhs; ++c) coef[(size_t)c] = active[(size_t)c] ? rz[(size_t)c] / h[(size_t)c] : 0.0;
      HM_CUDA(cudaMemcpyAsync(dscal, coef.data(), nrhs * sizeof(double), cudaMemcpyHostToDevice, st));
      HM_CUDA(launch_cg_xr(n, nrhs, dscal, P.as<double>(), Q.as<double>(), Xp.as<double>(), R.as<double>(), st));
      precond();
      dots(R, Z, 0);
      dots(R, R, 2);
      fetch();
      for (int64_t c = 0; c < nrhs; ++c) {
        coef[(size_t)c] = active[(size_t)c] ? h[(size_t)c] / rz[(size_t)c] : 0.0;
        if (active[(size_t)c]) {
          rz[(size_t)c] = h[(size_t)c];
          rr2[(size_t)c] = h[(size_t)(2 * nrhs + c)];
          iters[c] += 1;
        }
      }
      HM_CUDA(cudaMemcpyAsync(dscal + nrhs, coef.data(), nrhs * sizeof(double), cudaMemcpyHostToDevice, st));
      HM_CUDA(launch_cg_p(n, nrhs, dscal + nrhs, Z.as<double>(), P.as<double>(), st));
    }
    // true relative residuals ||b - A x|| / ||b||
    HM_CUDA(launch_csr_spmv(n, drp.as<int64_t>(), dci.as<int64_t>(), dva.as<double>(), Xp.as<double>(),
                            Q.as<double>(), nrhs, st));
    HM_CUDA(launch_sub(n * nrhs, Bp.as<double>(), Q.as<double>(), R.as<double>(), st));
    dots(R, R, 0);
    fetch();
    for (int64_t c = 0; c < nrhs; ++c)
      relres[c] = nb[(size_t)c] > 0.0 ? std::sqrt(h[(size_t)c]) / nb[(size_t)c] : 0.0;
    HM_CUDA(launch_permute(Xp.as<double>(), X, dperm.as<int64_t>(), n, nrhs, false, st));
    HM_CUDA(cudaStreamSynchronize(st));
  });
}

hmat_status trunc_lowrank(hmat_ctx* ctx, int64_t m, int64_t n, int64_t k, double* U, int64_t ldu, double* V,
                          int64_t ldv, double eps, int64_t* k_new) {
  return guarded([&] {
    check_ctx(ctx);
    require(U && V && k_new && ldu >= m && ldv >= n, "trunc_lowrank: bad arguments");
    require(ldu == std::max<int64_t>(m, 1) && ldv == std::max<int64_t>(n, 1), "trunc_lowrank: ld must equal the row count");
    DevBuf dk(sizeof(int64_t));
    double* Up = U;
    double* Vp = V;
    hmat_status s = trunc_lowrank_batched(ctx, 1, &m, &n, &k, &Up, &Vp, eps, dk.as<int64_t>(), HMAT_FP64, nullptr);
    if (s != HMAT_OK) throw HmError(s, g_last_error);
    HM_CUDA(cudaMemcpy(k_new, dk.p, sizeof(int64_t), cudaMemcpyDeviceToHost));
  });
}

hmat_status hmat_stats_get(const hmat* H, hmat_stats* out) {
  return guarded([&] {
    require(H && out, "null argument");
    hmat_stats s = H->st;
    std::vector<int> r((size_t)std::max(H->nslots, 1));
    HM_CUDA(cudaMemcpy(r.data(), H->ranks.p, (size_t)H->nslots * sizeof(int), cudaMemcpyDeviceToHost));
    int64_t mx = 0;
    double sum = 0;
    for (int i = 0; i < H->nslots; ++i) {
      mx = std::max<int64_t>(mx, r[(size_t)i]);
      sum += r[(size_t)i];
    }
    s.max_rank = mx;
    s.mean_rank = H->nslots ? sum / H->nslots : 0.0;
    *out = s;
  });
}

hmat_status hmat_lu_training_data(const hmat* H, int64_t max, float* X, float* y, int64_t* count) {
  return guarded([&] {
    require(H && count && (max <= 0 || (X && y)), "null argument");
    int64_t n = (int64_t)(H->train.size() / 7);
    *count = n;
    for (int64_t i = 0; i < std::min(n, max); ++i) {
      for (int j = 0; j < 6; ++j) X[i * 6 + j] = H->train[(size_t)(i * 7 + j)];
      y[i] = H->train[(size_t)(i * 7 + 6)];
    }
  });
}

hmat_status hmat_ranks(const hmat* H, int64_t* ranks) {
  return guarded([&] {
    require(H && ranks, "null argument");
    std::vector<int> r((size_t)std::max(H->nslots, 1));
    HM_CUDA(cudaMemcpy(r.data(), H->ranks.p, (size_t)H->nslots * sizeof(int), cudaMemcpyDeviceToHost));
    for (size_t b = 0; b < H->bt->nodes.size(); ++b)
      ranks[b] = H->bt->nodes[b].kind == 2 ? r[(size_t)H->slot[b]] : -1;
  });
}

}  // extern "C"

// Internal accessors for the other translation units of the library.
namespace hm_internal {
int ctx_device(const hmat_ctx* c) { return c->device; }
cudaStream_t ctx_stream(const hmat_ctx* c) { return c->stream; }
void set_last_error(const char* msg) { g_last_error = msg; }
}  // namespace hm_internal
