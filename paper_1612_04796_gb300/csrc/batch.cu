// Batched execution: several independent problems advance together, each
// sweep of the solver (operator, smoother, scatter, transfer, coarse pass,
// vector pass) issued as one grouped launch for all of them.
//
// The solver's launch sequence for one problem is recorded (launch_pdl with a
// recorder installed) instead of launched; the sequences of the problems are
// then merged: the records of one problem keep their order, and at each step
// one kernel found at the heads of the sequences (that of the sequence with
// the most records left) is launched once through its grouped twin
// (k_grouped) for every sequence that has it at its head, each problem
// getting its own block range and parameters; a launch with more blocks than
// the GPU holds at once runs the persistent form k_grouped_p (a grid of one
// wave looping over the problems' blocks; mg_opts.persistent).  Problems of different sizes, aspect ratios and even kernel
// variants (a small mesh takes the direction-split operator) merge as far as
// their sequences agree.
#include "mg_internal.h"

#include <algorithm>

namespace mgdg {

LaunchRecorder*& launch_recorder() {
  static thread_local LaunchRecorder* rec = nullptr;
  return rec;
}

namespace {

struct ScalarPtrs {
  const double* p[kMaxBatch];
};

__global__ void k_gather_scalars(ScalarPtrs src, int n, double* out) {
  const int i = threadIdx.x;
  if (i < n) out[i] = *src.p[i];
}

bool same_kernel(const LaunchRec& a, const LaunchRec& b) {
  return a.key == b.key && a.block.x == b.block.x && a.block.y == b.block.y && a.block.z == b.block.z &&
         a.smem == b.smem;
}

}  // namespace

cudaError_t launch_merged(const std::vector<LaunchRecorder>& seqs, cudaStream_t s, long long* launches, int persist) {
  const int B = (int)seqs.size();
  std::vector<size_t> head(B, 0);
  long long n_launch = 0;
  for (;;) {
    // The next kernel: the head of the sequence with the most records left
    // (ties: the head shared by the most sequences, then the lowest problem
    // index).  Sequences of different kernel variants differ by inserted
    // launches (a direction-split operator is three launches where the
    // element-block operator is one) and share their tails, so serving the
    // longest remaining sequence first brings them back into step at the
    // next common kernel instead of leaving one group behind.
    int best = -1, best_count = 0;
    size_t best_left = 0;
    for (int i = 0; i < B; ++i) {
      if (head[i] >= seqs[i].recs.size()) continue;
      const LaunchRec& r = seqs[i].recs[head[i]];
      int count = 0;
      size_t left = 0;
      for (int j = 0; j < B; ++j)
        if (head[j] < seqs[j].recs.size() && same_kernel(seqs[j].recs[head[j]], r)) {
          ++count;
          left = std::max(left, seqs[j].recs.size() - head[j]);
        }
      if (left > best_left || (left == best_left && count > best_count)) {
        best = i;
        best_count = count;
        best_left = left;
      }
    }
    if (best < 0) break;
    const LaunchRec& ref = seqs[best].recs[head[best]];
    const LaunchRec* group[kMaxBatch];
    int n = 0;
    for (int j = 0; j < B; ++j) {
      if (head[j] < seqs[j].recs.size() && same_kernel(seqs[j].recs[head[j]], ref)) {
        group[n++] = &seqs[j].recs[head[j]];
        ++head[j];
      }
    }
    cudaError_t e = cudaSuccess;
    if (ref.grouped) {  // a kernel with a body always runs its twin, also for one problem
      for (int k = 0; k < n && e == cudaSuccess; k += kMaxBatch) {
        e = ref.grouped(group + k, std::min(kMaxBatch, n - k), s, persist);
        ++n_launch;
      }
    } else {
      for (int k = 0; k < n && e == cudaSuccess; ++k) {
        e = group[k]->plain(*group[k], s);
        ++n_launch;
      }
    }
    if (e != cudaSuccess) return e;
  }
  if (launches) *launches += n_launch;
  return cudaGetLastError();
}

cudaError_t launch_gather_scalars(const double* const* src, int n, double* out, cudaStream_t s) {
  if (n < 1 || n > kMaxBatch) return cudaErrorInvalidValue;
  ScalarPtrs p{};
  for (int i = 0; i < n; ++i) p.p[i] = src[i];
  k_gather_scalars<<<1, 32, 0, s>>>(p, n, out);
  return cudaGetLastError();
}

}  // namespace mgdg
