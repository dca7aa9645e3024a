// The last kernel of a round captured as a CUDA graph: it publishes the
// round's sizes, swaps every derived relation's current and next versions
// (the ping-pong of full and delta buffers) and sets the condition of the
// graph's loop node, so that consecutive semi-naive rounds run on the device
// without the host (Section 3's loop: stop once no relation has a delta).
#include "kernels.h"

namespace cdl {

namespace {

__global__ void k_round_end(GraphRel* cur, GraphRel* next, uint32_t nrel, GraphCtl* ctl,
                            uint64_t* per_round, uint64_t per_round_cap,
                            cudaGraphConditionalHandle loop, uint64_t* cursors, uint32_t ncur,
                            uint64_t* steps, uint32_t nsteps) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (ctl->overflow) {  // cur holds the last complete round
    ctl->done = 2;
    cudaGraphSetConditional(loop, 0u);
    return;
  }
  uint64_t total = 0;
  for (uint32_t r = 0; r < nrel; ++r) {
    next[r].nF = cur[r].nF + next[r].nD;
    total += next[r].nD;
    const GraphRel t = cur[r];
    cur[r] = next[r];
    next[r] = t;
  }
  const uint64_t round = ++ctl->round;
  if (round - 1 < per_round_cap) per_round[round - 1] = total;
  if (total) ctl->iterations = round;
  if (total == 0)
    ctl->done = 1;
  else if (ctl->max_iters && ctl->iterations > ctl->max_iters)
    ctl->done = 3;
  for (uint32_t i = 0; i < ncur; ++i) cursors[i] = 0;  // the next round appends from 0
  for (uint32_t s = 0; s < nsteps; ++s) steps[3 * s + 2] = 0;
  cudaGraphSetConditional(loop, ctl->done ? 0u : 1u);
}

}  // namespace

cudaError_t round_end(Ctx& c, GraphRel* cur, GraphRel* next, uint32_t nrel, GraphCtl* ctl,
                      uint64_t* per_round, uint64_t per_round_cap,
                      cudaGraphConditionalHandle loop, uint64_t* cursors, uint32_t ncur,
                      uint64_t* steps, uint32_t nsteps) {
  k_round_end<<<1, 32, 0, c.st>>>(cur, next, nrel, ctl, per_round, per_round_cap, loop, cursors,
                                  ncur, steps, nsteps);
  return cudaGetLastError();
}

}  // namespace cdl
