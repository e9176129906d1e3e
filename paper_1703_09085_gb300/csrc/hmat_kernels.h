// hmat_kernels.h -- host-visible declarations of the device side.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "hmat_tasks.h"

namespace hm {

// Everything the persistent executor reads.
struct ExecEnv {
  double* hbase;              // H-matrix storage
  double* wsbase;             // workspace arena of this task list
  double* ext0;               // caller buffers addressed by tagged locations
  double* ext1;
  int* ranks;                 // rank slots
  const HTask* tasks;
  long long ntasks;
  const int64_t* dep_ptr;     // predecessors of task i: dep_idx[dep_ptr[i] .. dep_ptr[i+1])
  const int32_t* dep_idx;
  const LeafRef* leaves;
  int* done;                  // per task, 0 -> 1 when finished
  int* gang;                  // per task, the gang barrier counter of a gang's member 0
  unsigned long long* head;   // next task to take
  int* status;                // device status word (hmat_status numbering)
  long long* fail_task;       // 1 + index of the task that set the status first
  unsigned long long* counters;  // [0] truncations run, [1] randomised, [2] randomised fell back
  double* flops;              // FP64 operations counted by the tasks
  double* flops32;            // FP32 operations counted by the tasks (mixed path)
  double* bytes;              // algorithmic bytes of the tasks (what they must read and write)
  unsigned long long* type_ns;   // per task type: summed execution time (ns)
  unsigned long long* type_cnt;  // per task type: tasks run
  unsigned long long* wait_ns;   // summed time CTAs spent waiting on predecessors
  uint32_t* task_ns;             // optional: execution time of every task (profiling)
  uint32_t* task_aux;            // optional: truncation notes per task (profiling)
  const float* feat;             // 4 static features per task (truncations)
  const void* mlp;               // rank predictor weights (BF16), or null
  int oversample;                // sketch columns beyond the predicted rank
  float* rec;                    // optional: training pairs (7 floats each) of exact truncations
  unsigned long long* rec_count;
  long long rec_cap;
  double eps;
  int rank_rule;              // 0 relative Frobenius, 1 relative spectral (FP64 truncations)
  int mixed;                  // randomised truncation path on
  int rand_min_l;             // smallest stacked width that takes it
  unsigned long long seed;
  long long spin_iters;       // bounded waits: iteration limit
  unsigned long long spin_ns; //                 and time limit
};

struct TruncProblem {
  int m, n, k;
  int ldu, ldv;
  double* U;
  double* V;
  double* ws;       // (2m + n) k + 2 k^2 doubles
  int64_t* k_new;
};

struct DenseLeafDesc {
  int64_t off;      // offset of N in the H storage
  int64_t roff, coff;
  int rows, cols;
};

size_t smem_bytes();
cudaError_t exec_occupancy(int* blocks_per_sm);
cudaError_t launch_exec(const ExecEnv& env, int grid, cudaStream_t st);
cudaError_t launch_trunc_batched(const TruncProblem* probs, int count, double eps, int* status, int mixed,
                                 cudaStream_t st);
cudaError_t launch_csr_scatter(const DenseLeafDesc* leaves, int nleaves, const int64_t* rowptr,
                               const int64_t* colidx, const double* val, const int64_t* perm, const int64_t* iperm,
                               double* hbase, unsigned long long* placed, cudaStream_t st);
// Conjugate-gradient building blocks on n x nrhs column-major blocks (ld n).
// dst(i, c) = src(perm[i], c) (gather) or dst(perm[i], c) = src(i, c).
cudaError_t launch_permute(const double* src, double* dst, const int64_t* perm, int64_t n, int64_t nrhs, bool gather,
                           cudaStream_t st);
// Y = A X with A in CSR form (row pointers, column indices, values).
cudaError_t launch_csr_spmv(int64_t n, const int64_t* rowptr, const int64_t* colidx, const double* val,
                            const double* X, double* Y, int64_t nrhs, cudaStream_t st);
// out[c] = sum_i X(i, c) Y(i, c).
cudaError_t launch_col_dots(int64_t n, int64_t nrhs, const double* X, const double* Y, double* out, cudaStream_t st);
// X += alpha[c] P, R -= alpha[c] Q (per column c).
cudaError_t launch_cg_xr(int64_t n, int64_t nrhs, const double* alpha, const double* P, const double* Q, double* X,
                         double* R, cudaStream_t st);
// P = Z + beta[c] P; or, with D given, D = B - Q.
cudaError_t launch_cg_p(int64_t n, int64_t nrhs, const double* beta, const double* Z, double* P, cudaStream_t st);
cudaError_t launch_sub(int64_t count, const double* A, const double* B, double* D, cudaStream_t st);
cudaError_t launch_to_dense(const LeafRef* leaves, int nleaves, const double* hbase, const int* ranks, double* out,
                            int64_t ldo, cudaStream_t st);

}  // namespace hm
