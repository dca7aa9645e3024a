// Retirement of converged instances inside a captured round (batched runs,
// option graph).  An instance that derived nothing in the round just ended
// has reached its own fixpoint: instances share no tuples and every rule
// joins on the instance column.  Once the rows of such instances waiting to
// leave reach 1/8 of the derived relations' rows, they move from Full to a
// retired buffer, so that later rounds merge only the instances still
// running.  The host version of this pass builds the segment tables on the
// host; here every decision and table is made on the device, after the
// round's last kernel (k_round_end), so that the rounds keep running inside
// the graph's loop:
//   k_retire_bounds  -- per relation, the first row of every instance in
//                       Full (sorted with the instance id in column 0);
//   k_retire_plan    -- one block: marks newly converged instances, decides
//                       whether rows move this round, and builds, per
//                       relation, the table of kept segments and the table of
//                       retired segments (one per instance, empty ones
//                       included) and the instances' places in the retired
//                       buffer;
//   k_retire_gather  -- kept rows into the free half of Full's ping-pong
//                       pair, retired rows appended to the retired buffer;
//   k_retire_commit  -- the kept rows become Full.
// Every kernel reads the decision from device memory and does nothing when
// no rows move.
#include "kernels.h"

namespace cdl {

namespace {

constexpr int kPlanT = 1024;
constexpr int kGatherT = 256;

__global__ void k_retire_bounds(const GraphRel* cur, uint32_t j, uint32_t ni, RetireRel* rr) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i > ni) return;
  const uint32_t* inst = cur[j].F.c[0];
  uint64_t lo = 0, hi = cur[j].nF;
  while (lo < hi) {
    const uint64_t mid = (lo + hi) >> 1;
    if ((uint64_t)__ldg(inst + mid) < i)
      lo = mid + 1;
    else
      hi = mid;
  }
  rr[j].bounds[i] = lo;
}

// Block-wide exclusive sum of v over the block; total in *tot.
__device__ __forceinline__ uint64_t plan_scan(uint64_t v, uint64_t* red, uint64_t* tot) {
  return block_exclusive_sum<kPlanT, uint64_t>(v, red, tot);
}

__global__ void __launch_bounds__(kPlanT) k_retire_plan(const GraphRel* cur, GraphCtl* ctl,
                                                        RetireCtl* rc, RetireRel* rr,
                                                        uint32_t nrel, uint32_t ni,
                                                        const uint64_t* last_round) {
  __shared__ uint64_t red[kPlanT / 32 + 1];
  __shared__ uint64_t s_wait, s_rows;
  __shared__ uint32_t s_go;
  const uint32_t t = threadIdx.x;
  if (t == 0) {
    s_wait = s_rows = 0;
    rc->go = 0;
  }
  __syncthreads();
  if (ctl->done == 2) return;  // the round did not complete: nothing moves
  const uint64_t round = ctl->round;
  // newly converged instances: running, and no new tuple in this round
  for (uint32_t i = t; i < ni; i += kPlanT)
    if (rc->live[i] && !rc->conv[i] && last_round[i] != round) rc->conv[i] = 1;
  __syncthreads();
  uint64_t wait = 0;
  for (uint32_t j = 0; j < nrel; ++j)
    for (uint32_t i = t; i < ni; i += kPlanT)
      if (rc->live[i] && rc->conv[i]) wait += rr[j].bounds[i + 1] - rr[j].bounds[i];
  atomicAdd(reinterpret_cast<unsigned long long*>(&s_wait), (unsigned long long)wait);
  if (t == 0) {
    uint64_t rows = 0;
    for (uint32_t j = 0; j < nrel; ++j) rows += cur[j].nF;
    s_rows = rows;
  }
  __syncthreads();
  if (t == 0) {
    bool go = s_wait > 0 && s_wait * 8 >= s_rows;
    for (uint32_t j = 0; j < nrel && go; ++j) {  // room in every retired buffer
      uint64_t out = 0;
      for (uint32_t i = 0; i < ni; ++i)
        if (rc->live[i] && rc->conv[i]) out += rr[j].bounds[i + 1] - rr[j].bounds[i];
      if (rr[j].ret_n + out > rr[j].ret_cap) {
        go = false;
        rc->short_room = 1;  // the host gives the next graph more room
      }
    }
    s_go = go ? 1u : 0u;
  }
  __syncthreads();
  if (!s_go) return;
  for (uint32_t j = 0; j < nrel; ++j) {
    RetireRel& R = rr[j];
    uint64_t kcarry = 0, rcarry = R.ret_n;
    for (uint32_t i0 = 0; i0 < ni; i0 += kPlanT) {
      const uint32_t i = i0 + t;
      uint64_t kl = 0, rl = 0, b = 0;
      if (i < ni) {
        b = R.bounds[i];
        const uint64_t cnt = R.bounds[i + 1] - b;
        if (rc->live[i]) (rc->conv[i] ? rl : kl) = cnt;
      }
      uint64_t ktot, rtot;
      const uint64_t kx = plan_scan(kl, red, &ktot);
      const uint64_t rx = plan_scan(rl, red, &rtot);
      if (i < ni) {
        R.kseg_off[i] = kcarry + kx;
        R.kseg_src[i] = b;
        R.rseg_off[i] = rcarry + rx;
        R.rseg_src[i] = b;
        if (rl) {
          R.ret_off[i] = rcarry + rx;
          R.ret_cnt[i] = rl;
        }
      }
      kcarry += ktot;
      rcarry += rtot;
    }
    if (t == 0) {
      R.kseg_off[ni] = kcarry;
      R.rseg_off[ni] = rcarry;
      R.kept = kcarry;
      R.moved = rcarry - R.ret_n;
    }
    __syncthreads();
  }
  for (uint32_t i = t; i < ni; i += kPlanT)
    if (rc->live[i] && rc->conv[i]) rc->live[i] = 0;
  if (t == 0) rc->go = 1;
}

// Output rows [off[s], off[s + 1]) copy source rows src[s] ...; the segment
// of output row j by binary search over the ni + 1 offsets.
__device__ __forceinline__ void gather_rows(const ColsIn& from, uint32_t k, ColsOut to,
                                            uint64_t first, uint64_t end, const uint64_t* off,
                                            const uint64_t* src, uint32_t ni) {
  for (uint64_t j = first + (uint64_t)blockIdx.x * kGatherT + threadIdx.x; j < end;
       j += (uint64_t)gridDim.x * kGatherT) {
    uint32_t lo = 0, hi = ni;  // the last segment whose start is <= j
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (__ldg(off + mid) <= j)
        lo = mid;
      else
        hi = mid;
    }
    const uint64_t row = __ldg(src + lo) + (j - __ldg(off + lo));
    for (uint32_t c = 0; c < k; ++c) to.c[c][j] = __ldg(from.c[c] + row);
  }
}

__global__ void __launch_bounds__(kGatherT) k_retire_gather(const GraphRel* cur,
                                                            const GraphRel* next, uint32_t j,
                                                            uint32_t k, const RetireCtl* rc,
                                                            const RetireRel* rr, uint32_t ni) {
  if (!rc->go) return;
  const RetireRel& R = rr[j];
  ColsOut kept;
  for (int c = 0; c < kMaxK; ++c) kept.c[c] = const_cast<uint32_t*>(next[j].F.c[c]);
  gather_rows(cur[j].F, k, kept, 0, R.kept, R.kseg_off, R.kseg_src, ni);
  gather_rows(cur[j].F, k, R.ret, R.ret_n, R.ret_n + R.moved, R.rseg_off, R.rseg_src, ni);
}

__global__ void k_retire_commit(GraphRel* cur, GraphRel* next, uint32_t nrel, RetireCtl* rc,
                                RetireRel* rr) {
  if (threadIdx.x != 0 || blockIdx.x != 0 || !rc->go) return;
  ++rc->moves;
  for (uint32_t j = 0; j < nrel; ++j) {
    const ColsIn t = cur[j].F;
    cur[j].F = next[j].F;
    next[j].F = t;
    cur[j].nF = rr[j].kept;
    rr[j].ret_n += rr[j].moved;
  }
}

}  // namespace

cudaError_t retire_round(Ctx& c, GraphRel* cur, GraphRel* next, GraphCtl* ctl, RetireCtl* rc,
                         RetireRel* rr, const uint32_t* arity, uint32_t nrel, uint32_t ni,
                         const uint64_t* last_round) {
  ProfScope p(c, kRetire, 0.0);
  for (uint32_t j = 0; j < nrel; ++j)
    k_retire_bounds<<<(ni + 256) / 256, 256, 0, c.st>>>(cur, j, ni, rr);
  k_retire_plan<<<1, kPlanT, 0, c.st>>>(cur, ctl, rc, rr, nrel, ni, last_round);
  for (uint32_t j = 0; j < nrel; ++j)
    k_retire_gather<<<152 * 8, kGatherT, 0, c.st>>>(cur, next, j, arity[j], rc, rr, ni);
  k_retire_commit<<<1, 32, 0, c.st>>>(cur, next, nrel, rc, rr);
  return cudaGetLastError();
}

}  // namespace cdl
