// persist.cuh -- one persistent launch for every sweep of a batch.
//
// The jobs of a batch (Eq. 4's N_alpha realizations) are independent; the
// sweeps of one job are not: sweep i of a job reads what every tile of its
// sweep i - 1 wrote.  persist_kernel's blocks pull work items -- one tile of
// one sweep of one job -- from a device queue (an atomic counter) in the
// order (sweep index, group, job, tile), and before working on an item wait
// until every tile of the job's earlier sweeps is done (a per-job counter).
// Every item an item waits on comes earlier in the queue, so it is held by a
// running block or finished: the waits always end.  They are bounded all the
// same: a wait that exceeds kPersistWaitLimit polls sets the launch's error
// word, and every block then stops taking items and returns.
#pragma once
#include "kernels.cuh"

namespace spinrp {

constexpr int kMaxPersistGroups = 16;
constexpr int kMaxSteadyPasses = 64;
constexpr unsigned kPersistWaitLimit = 1u << 21;  // polls, each an L2 round trip and a short sleep: about a second

struct PersistGroup {
  int M, K;
  int njobs;
  int done0;                    // this group's first counter in the done array
  int nsweeps;                  // sweeps of the evolve call: 1 + S * steps
  int S;                        // sweeps per Trotter step
  int head, join, tail;         // pass indices into `passes`
  int steady[kMaxSteadyPasses];  // passes 0..S-2 of a step (body, middle, reverse body)
  unsigned tiles;               // tiles per sweep, 2^(M - K)
  int pad;
  unsigned long long cum;       // items of the groups before this one, per sweep index
  const PassDesc *passes;
  const PhaseDesc *phases;
  const JobPtrs *jobs;          // the group's job table
};

// Groups are sorted by nsweeps, most first; region k covers the sweep indices
// [start[k], start[k + 1]) in which the first active[k] groups still have
// sweeps, per[k] items per sweep index from item base[k] on.
struct PersistPlan {
  int ngroups, nregions;
  long long steps;
  unsigned long long total;
  int start[kMaxPersistGroups + 1];
  int active[kMaxPersistGroups];
  unsigned long long base[kMaxPersistGroups];
  unsigned long long per[kMaxPersistGroups];
  PersistGroup g[kMaxPersistGroups];
};

namespace pq {

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_relaxed(const int *p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
// 8-byte load through L2 only: tiles written by other SMs earlier in the
// same launch are read from the coherent level, never from a stale L1 line.
__device__ __forceinline__ float2 ld_cg(const float2 *p) {
  float2 v;
  asm volatile("ld.global.cg.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
  return v;
}

// Global -> shared copy of a tile as sw2::load_tile walks it, through
// registers with L2-only loads.
template <int RB>
__device__ __forceinline__ void load_tile_cg(const float2 *psi, uint64_t base, const PassDesc &d, int tid,
                                             int lognt, float2 *tile2) {
  constexpr int NA = 1 << RB;
  uint64_t off_amp_lo = 0;
  for (int k = 0; k < lognt; ++k)
    if ((tid >> k) & 1) off_amp_lo |= 1ull << d.tile_pos[k];
  int64_t dg[RB];
  uint32_t ds[RB];
#pragma unroll
  for (int k = 0; k < RB; ++k) {
    dg[k] = (int64_t)1 << d.tile_pos[lognt + k];
    ds[k] = sw2::slot(1u << (lognt + k));
  }
  const float2 *src0 = psi + base + off_amp_lo;
  const uint32_t sb0 = sw2::slot((uint32_t)tid);
  // every load first (one round trip), then the shared-memory stores, their
  // slots walked again
  float2 v[NA];
  const float2 *src = src0;
#pragma unroll
  for (int g = 0; g < NA; ++g) {
    if ((g & 7) == 0) {
      src = src0;
#pragma unroll
      for (int k = 0; k < RB; ++k)
        if (((g ^ (g >> 1)) >> k) & 1) src += dg[k];
    } else {
      const int k = sw2::ctz6(g);
      src += sw2::gray_up(g) ? dg[k] : -dg[k];
    }
    v[g] = ld_cg(src);
  }
  uint32_t sb = sb0;
#pragma unroll
  for (int g = 0; g < NA; ++g) {
    if ((g & 7) == 0) {
      sb = sb0;
#pragma unroll
      for (int k = 0; k < RB; ++k)
        if (((g ^ (g >> 1)) >> k) & 1) sb ^= ds[k];
    } else {
      sb ^= ds[sw2::ctz6(g)];
    }
    tile2[sb] = v[g];
  }
}

// Per-job grid reduction of one reducing sweep inside the persistent launch:
// as reduce_finalize, with the tile index r of ntiles in place of the block
// index; every thread of the block calls it.
__device__ void reduce_tile(double up, double dn, const JobPtrs &jp, unsigned r, unsigned ntiles,
                            double *s_up, double *s_dn, int *s_last) {
  for (int o = 16; o; o >>= 1) {
    up += __shfl_xor_sync(0xffffffffu, up, o);
    dn += __shfl_xor_sync(0xffffffffu, dn, o);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (lane == 0) s_up[warp] = up, s_dn[warp] = dn;
  __syncthreads();
  if (threadIdx.x == 0) {
    double u = 0.0, d = 0.0;
    for (int w = 0; w < nw; ++w) u += s_up[w], d += s_dn[w];
    jp.partials[r] = make_double2(u, d);
    __threadfence();
    *s_last = atomicAdd(jp.ticket, 1u) == ntiles - 1;
  }
  __syncthreads();
  if (*s_last) {
    __threadfence();
    double u = 0.0, d = 0.0;
    for (unsigned b = threadIdx.x; b < ntiles; b += blockDim.x) {
      const double2 p = __ldcg(&jp.partials[b]);
      u += p.x, d += p.y;
    }
    for (int o = 16; o; o >>= 1) {
      u += __shfl_xor_sync(0xffffffffu, u, o);
      d += __shfl_xor_sync(0xffffffffu, d, o);
    }
    __syncthreads();
    if (lane == 0) s_up[warp] = u, s_dn[warp] = d;
    __syncthreads();
    if (threadIdx.x == 0) {
      double U = 0.0, D = 0.0;
      for (int w = 0; w < nw; ++w) U += s_up[w], D += s_dn[w];
      const int64_t slot = __ldcg(jp.step);  // written earlier in this launch, maybe by another SM
      jp.series[2 * slot] = (U - D) / (U + D);
      jp.series[2 * slot + 1] = U + D;
      *jp.step = slot + 1;
      *jp.ticket = 0u;
    }
  }
  __syncthreads();
}

}  // namespace pq

// 2^(K-RB) threads per block, K the same for every group of the launch (13
// or 14); dynamic shared memory: one 2^K tile.  queue: item counter, done:
// per-job finished tiles of this launch, err: nonzero after a wait timed out
// (all cleared before the launch).
template <int RB>
__global__ void __launch_bounds__(256)
persist_kernel(const PersistPlan *__restrict__ plan, unsigned long long *queue, unsigned *done, int *err,
               unsigned ahead) {
  extern __shared__ __align__(16) float2 tile2[];
  __shared__ uint64_t sH[kMaxK];
  __shared__ uint64_t sQ[kMaxK * kMaxK];
  __shared__ uint64_t sOut;
  __shared__ __align__(16) PhaseDesc s_ph[kMaxPassPhases];
  __shared__ __align__(16) ROpRes s_op[kMaxPassOps];
  __shared__ __align__(16) PassDesc s_d;
  __shared__ double s_up[8], s_dn[8];
  __shared__ unsigned long long s_item;
  __shared__ int s_go, s_last;
  const int tid = threadIdx.x, nt = blockDim.x;
  const unsigned long long total = plan->total;
  // thread 0 decodes an item into (sweep index, group, job, pass, tile); the
  // next item is taken from the queue while the current one computes
  struct Item {
    int i, gi, jl, pass;
    unsigned r;
  };
  __shared__ Item s_it;
  auto decode = [&](unsigned long long x) -> Item {
    Item it;
    int k = 0;
    while (k + 1 < plan->nregions && x >= plan->base[k + 1]) ++k;
    const unsigned long long off = x - plan->base[k];
    const unsigned per = (unsigned)plan->per[k];  // < 2^32 (host check)
    const unsigned long long q0 = off / per;
    it.i = plan->start[k] + (int)q0;
    const unsigned rem = (unsigned)(off - q0 * per);
    int gi = 0;
    while (gi + 1 < plan->active[k] && rem >= plan->g[gi + 1].cum) ++gi;
    const PersistGroup &G = plan->g[gi];
    const unsigned w = rem - (unsigned)G.cum;
    it.gi = gi;
    it.jl = (int)(w / G.tiles);
    it.r = w - (unsigned)it.jl * G.tiles;
    if (it.i == 0) {
      it.pass = G.head;
    } else {
      const int q = (it.i - 1) % G.S;
      const long long step = (it.i - 1) / G.S;
      it.pass = q < G.S - 1 ? G.steady[q] : (step == plan->steps - 1 ? G.tail : G.join);
    }
    return it;
  };
  unsigned long long next = 0;
  if (tid == 0) next = atomicAdd(queue, 1ull);
  for (;;) {
    if (tid == 0) {
      s_item = next;
      s_go = next < total;
      if (s_go) {
        const Item it = decode(next);
        s_it = it;
        // the job's earlier sweeps, every tile of them, must be done
        const PersistGroup &G = plan->g[it.gi];
        const unsigned need = (unsigned)it.i * G.tiles;
        unsigned polls = 0;
        while (pq::ld_acquire(done + G.done0 + it.jl) < need) {
          if (++polls > kPersistWaitLimit || pq::ld_relaxed(err)) {
            atomicExch(err, 1);
            s_go = 0;
            break;
          }
          __nanosleep(100);
        }
      }
    }
    __syncthreads();
    if (!s_go) break;
    const Item it = s_it;
    const PersistGroup &G = plan->g[it.gi];
    const int jl = it.jl, pass = it.pass;
    const unsigned r = it.r;
    // the pass descriptor
    {
      const int nwords = (int)(sizeof(PassDesc) / 4);
      const int *src = reinterpret_cast<const int *>(G.passes + pass);
      for (int q = tid; q < nwords; q += nt) reinterpret_cast<int *>(&s_d)[q] = src[q];
    }
    __syncthreads();
    const PassDesc &d = s_d;
    const JobPtrs jp = G.jobs[jl];
    float2 *__restrict__ psi = static_cast<float2 *>(jp.psi);
    const int lognt = d.K - RB, M = G.M;
    const uint64_t base = sw2::tile_origin(r, d, M);
    {
      const uint32_t *pw = reinterpret_cast<const uint32_t *>(G.phases + d.phase0);
      const uint32_t a_ph = (uint32_t)__cvta_generic_to_shared(s_ph);
      const int nw = d.nphases * (int)(sizeof(PhaseDesc) / 4);
      for (int q = tid; q < nw; q += nt) sw2::cp_async4(a_ph + 4u * q, pw + q);
      const ROpRes *so = jp.sops + d.rop0;
      const uint32_t a_op = (uint32_t)__cvta_generic_to_shared(s_op);
      for (int q = tid; q < d.nrops; q += nt) sw2::cp_async16(a_op + 16u * q, so + q);
    }
    // L2 prefetch of the tile `ahead` items on, when it is a tile of the same
    // job's same sweep
    if (ahead && r + ahead < G.tiles) sw2::prefetch_tile<RB>(psi, sw2::tile_origin(r + ahead, d, M), d, tid, lognt);
    pq::load_tile_cg<RB>(psi, base, d, tid, lognt, tile2);
    if (tid == 0) next = atomicAdd(queue, 1ull);
    sw2::cp_async_wait_all();
    __syncthreads();
    float up = 0.f, dn = 0.f;
    sw2::run_phases<RB, false, false>(tile2, d, s_ph, s_op, base, tid, lognt, M, jp.qdiag, up, dn, sH, sQ,
                                      &sOut, nullptr, sw2::SyncBlock{});
    sw2::store_tile<RB>(psi, base, d, tid, lognt, tile2);
    if (d.has_reduce) pq::reduce_tile((double)up, (double)dn, jp, r, G.tiles, s_up, s_dn, &s_last);
    __threadfence();
    __syncthreads();
    if (tid == 0) atomicAdd(done + G.done0 + jl, 1u);
  }
}

}  // namespace spinrp
