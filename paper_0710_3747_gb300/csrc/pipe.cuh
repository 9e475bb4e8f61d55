// pipe.cuh -- a sweep as one persistent, warp-specialised launch.
//
// sweep2_kernel gives every tile its own block: gather the tile into shared
// memory, run the register-blocked phases, write it back.  Two blocks share an
// SM, and one block's copies overlap the other's phases only as far as the
// warp scheduler happens to interleave them; the copy time mostly adds to
// the phase time.  pipe_kernel runs one block per SM for the whole sweep and
// gives its warps fixed roles:
//
//   * a producer warpgroup (128 threads) moves tiles between global and
//     shared memory: the 8-byte asynchronous gathers of sw2::load_tile and the
//     coalesced 16-byte stores of sw2::store_tile;
//   * two compute warpgroups of 2^(K-RB) = 128 threads run sw2::run_phases,
//     each on its own tile, each synchronised by its own named barrier.
//
// The register file is split per SM sub-partition, and each of the four holds
// one warp of every warpgroup.  The block is launched at 168 registers a
// thread (3 x 128 x 168 = 64512); the producer gives registers back
// (setmaxnreg.dec to 56) and the compute groups take them (setmaxnreg.inc to
// 224, what the phases need without spilling): 128 x 56 + 256 x 224 = 64512.
//
// Three tile buffers rotate through load -> phases -> store.  Block b takes
// the units b, b + G, b + 2G, ... (G blocks; a unit is a tile, or for a batch
// one job's tile), local unit i in buffer i mod 3 and in group i mod 2;
// shared-memory mbarriers hand a buffer over: full[k]
// completes when the producer's copies of the tile in buffer k have landed
// (cp.async arrive-on), done[k] when a group has finished its phases on it.
// While the groups compute two tiles, the producer writes back the previous
// one, gathers the next and prefetches the one after into L2.
//
// Every amplitude goes through the same floating-point operations in the
// same order as in sweep2_kernel, each tile's (N_up, N_dn) partial is summed
// the same way, and a job's partials are combined in tile order the way
// reduce_finalize combines block partials (one job: by the last block to
// finish; a batch: by pipe_finalize_kernel): the results are the same bit
// for bit.
//
// Waits are bounded by the global timer (kPipeWaitNs).  A wait that runs out
// sets the error word; the block's other waits then run out too, the
// producer waits for its own copies in flight, every thread leaves its loop,
// and the reducing sweep records NaN for P and the norm.  Named barriers: 0
// the whole block (prologue only), 1 and 2 the compute groups, 3 the
// producer, 4 both compute groups.
#pragma once
#include "kernels.cuh"

namespace spinrp {

constexpr unsigned long long kPipeWaitNs = 2000000000ull;  // 2 s

namespace pipe {

__device__ __forceinline__ uint64_t now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(bar) : "memory");
}
// The barrier tracks the completion of this thread's earlier cp.async copies;
// the arrival counts towards the expected count (noinc).
__device__ __forceinline__ void cp_async_arrive(uint32_t bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase of parity `parity` to complete, at most kPipeWaitNs, and
// give up early once the error word is set; false when the wait gave up.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, const int *err) {
  if (mbar_test(bar, parity)) return true;
  const uint64_t t0 = now_ns();
  for (unsigned n = 1;; ++n) {
    if (mbar_test(bar, parity)) return true;
    if ((n & 63u) == 0) {
      if (now_ns() - t0 > kPipeWaitNs) return false;
      if (*(volatile const int *)err) return false;
    }
  }
}
// Barrier of a compute group (named barrier `id`, n threads) ...
struct SyncNamed {
  uint32_t id, n;
  __device__ __forceinline__ void operator()() const {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
  }
};
// ... and the same barrier with an OR over the group's predicates.
__device__ __forceinline__ bool group_any(bool v, uint32_t id, uint32_t n) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbarrier.red.or.pred q, %2, %3, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)v), "r"(id), "r"(n)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void cp_async_drain() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

}  // namespace pipe

constexpr int kPipeThreads = 384;  // two compute warpgroups and a producer warpgroup
constexpr int kPipeRegsCompute = 224;
constexpr int kPipeRegsProducer = 56;
static_assert(2 * 128 * kPipeRegsCompute + 128 * kPipeRegsProducer <= kPipeThreads * 168,
              "register split above the launch's registers");

// Sum of a job's T tile partials in tile order by the 128 threads t of a
// group (barrier `sync`), the order reduce_finalize uses for a 128-thread
// block; thread 0 appends (P, norm) -- NaN after a wait gave up -- at the
// job's step counter and advances it.  Scratch su/sd: the group's NW doubles.
template <int NW, typename Sync>
__device__ __forceinline__ void pipe_finalize(const double2 *partials, unsigned *ticket, int64_t *step,
                                              double *series, unsigned T, int t, const int *err, double *su,
                                              double *sd, Sync sync) {
  double u = 0.0, v = 0.0;
  for (unsigned b = (unsigned)t; b < T; b += 32u * NW) {
    const double2 p = __ldcg(&partials[b]);
    u += p.x, v += p.y;
  }
  for (int o = 16; o; o >>= 1) {
    u += __shfl_xor_sync(0xffffffffu, u, o);
    v += __shfl_xor_sync(0xffffffffu, v, o);
  }
  if ((t & 31) == 0) su[t >> 5] = u, sd[t >> 5] = v;
  sync();
  if (t == 0) {
    double U = 0.0, D = 0.0;
    for (int w = 0; w < NW; ++w) U += su[w], D += sd[w];
    const bool bad = *(volatile const int *)err != 0;
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    const int64_t slot = *step;
    series[2 * slot] = bad ? nan : (U - D) / (U + D);
    series[2 * slot + 1] = bad ? nan : U + D;
    *step = slot + 1;
    *ticket = 0u;
  }
}

// One sweep (complex64, plain storage, spin-1 readout) with 2^(K-RB) = 128
// threads per compute group.  (A sweep that takes the all-site readout runs
// sweep2_kernel's readout variant: under this kernel's 224-register budget
// the readout's sums spill, measured 8 % slower per step at M = 30.)
//   BATCH = false: one job; jobs[0] holds its pointers (gate tables,
//     partials, ticket, series), psi1 and sops1 its amplitudes and resolved
//     ops; the units are its tiles, and the last block to finish combines
//     the tile partials.
//   BATCH = true: njobs jobs of the same plan (jobs[j]), job j's amplitudes
//     and resolved ops at psi1 and sops1 plus j x jstride bytes; the units
//     are the (job, tile) pairs, job-major; the producer copies each unit's job
//     pointers and resolved ops (at most kPipeBatchOps) into its buffer's
//     slots of static shared arrays with the tile (the same mbarrier covers
//     them); each tile leaves its partial, and pipe_finalize_kernel,
//     launched after a reducing sweep, combines every job's partials.
// err: the error word.  probe: the producer issues no copies, so every wait
// runs out (the check that the waits are bounded; nothing is written to the
// amplitudes or the series).  Dynamic shared memory: three 8 x 2^K byte tile
// buffers.
constexpr int kPipeBatchOps = kMaxPassOps / 3;  // resolved ops of a pass, per buffer (batches)
static_assert(sizeof(JobPtrs) % 8 == 0, "job pointers copied as 8-byte words");

template <int RB, int K, bool BATCH>
__global__ void __launch_bounds__(kPipeThreads, 1)
pipe_kernel(const JobPtrs *__restrict__ jobs, int njobs, float2 *psi1, const ROpRes *sops1, long long jstride,
            const __grid_constant__ PassDesc d, const PhaseDesc *__restrict__ phases, int M, int *err, int probe) {
  constexpr int LOGNT = K - RB;
  constexpr int NT = 1 << LOGNT;   // threads of a group (a warpgroup)
  constexpr int NW = NT / 32;      // warps of a group
  constexpr uint32_t TA = 1u << K; // amplitudes per tile buffer
  static_assert(NT == 128, "groups are warpgroups");
  extern __shared__ __align__(16) float2 tiles[];
  __shared__ uint64_t sH[2][kMaxK];
  __shared__ uint64_t sQ[2][kMaxK * kMaxK];
  __shared__ uint64_t sOut[2];
  __shared__ __align__(16) PhaseDesc s_ph[kMaxPassPhases];
  // one job: the pass's ops; BATCH: three slices of kPipeBatchOps, one per buffer
  __shared__ __align__(16) ROpRes s_op[kMaxPassOps];
  __shared__ __align__(16) JobPtrs s_job[BATCH ? 3 : 1];
  __shared__ __align__(8) uint64_t s_full[3], s_done[3];
  __shared__ double s_up[2][NW], s_dn[2][NW];
  __shared__ int s_last;

  const int tid = threadIdx.x;
  const unsigned G = gridDim.x;
  const int lt = M - K;                       // log2 tiles per job
  const unsigned T = 1u << lt;
  const unsigned nunits = BATCH ? (unsigned)njobs << lt : T;
  const unsigned nloc = blockIdx.x < nunits ? (nunits - 1u - blockIdx.x) / G + 1u : 0u;
  const uint32_t a_tiles = (uint32_t)__cvta_generic_to_shared(tiles);
  const uint32_t a_full = (uint32_t)__cvta_generic_to_shared(s_full);
  const uint32_t a_done = (uint32_t)__cvta_generic_to_shared(s_done);
  const uint32_t a_jobs = (uint32_t)__cvta_generic_to_shared(s_job);
  const uint32_t a_ops = (uint32_t)__cvta_generic_to_shared(s_op);

  // the pass's program, once for the whole sweep (one job: its ops too)
  {
    const uint32_t *pw = reinterpret_cast<const uint32_t *>(phases + d.phase0);
    const uint32_t a_ph = (uint32_t)__cvta_generic_to_shared(s_ph);
    const int nw = d.nphases * (int)(sizeof(PhaseDesc) / 4);
    for (int i = tid; i < nw; i += kPipeThreads) sw2::cp_async4(a_ph + 4u * i, pw + i);
    if (!BATCH) {
      const uint32_t a_op = (uint32_t)__cvta_generic_to_shared(s_op);
      for (int i = tid; i < d.nrops; i += kPipeThreads) sw2::cp_async16(a_op + 16u * i, sops1 + d.rop0 + i);
    }
  }
  if (tid == 0)
    for (int k = 0; k < 3; ++k) {
      pipe::mbar_init(a_full + 8u * k, (unsigned)NT);
      pipe::mbar_init(a_done + 8u * k, 1u);
    }
  sw2::cp_async_wait_all();
  __syncthreads();

  if (tid >= 2 * NT) {
    // producer: at step i write back local unit i - 3, then gather unit i
    // into the buffer it left (i mod 3) and prefetch unit i + 1 into L2
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kPipeRegsProducer));
    const int pt = tid - 2 * NT;
    auto amps = [&](unsigned u) -> float2 * {
      return BATCH ? reinterpret_cast<float2 *>(reinterpret_cast<char *>(psi1) + (long long)(u >> lt) * jstride)
                   : psi1;
    };
    bool ok = true;
    for (unsigned i = 0; i < nloc + 3u; ++i) {
      const uint32_t b = i % 3u;
      if (i >= 3u) {
        const unsigned u = blockIdx.x + (i - 3u) * G;
        const bool late = !pipe::mbar_wait(a_done + 8u * b, ((i - 3u) / 3u) & 1u, err);
        if (pipe::group_any(late, 3u, NT)) {  // one outcome for the group
          ok = false;
          break;
        }
        sw2::store_tile<RB>(amps(u), sw2::tile_origin(u & (T - 1u), d, M), d, pt, LOGNT, tiles + b * TA);
        pipe::SyncNamed{3u, (uint32_t)NT}();  // every read of the buffer before its refill
      }
      if (i < nloc && !probe) {
        const unsigned u = blockIdx.x + i * G;
        if (BATCH) {
          // the unit's job pointers and ops beside its tile
          const JobPtrs *src = jobs + (u >> lt);
          if (pt < (int)(sizeof(JobPtrs) / 8))
            sw2::cp_async8(a_jobs + (uint32_t)sizeof(JobPtrs) * b + 8u * pt, reinterpret_cast<const char *>(src) + 8 * pt);
          const ROpRes *so =
              reinterpret_cast<const ROpRes *>(reinterpret_cast<const char *>(sops1) + (long long)(u >> lt) * jstride) +
              d.rop0;
          const uint32_t ab = a_ops + 16u * (uint32_t)kPipeBatchOps * b;
          for (int w = pt; w < d.nrops; w += NT) sw2::cp_async16(ab + 16u * w, so + w);
        }
        sw2::load_tile<RB>(amps(u), sw2::tile_origin(u & (T - 1u), d, M), d, pt, LOGNT, a_tiles + 8u * TA * b);
        pipe::cp_async_arrive(a_full + 8u * b);
        // unit i + 1 into L2 while unit i - 2 computes: its gather at the
        // next step then reads L2 (measured: one unit ahead beats two, three
        // or none)
        if (i + 1u < nloc) {
          const unsigned u1 = u + G;
          sw2::prefetch_tile<RB>(amps(u1), sw2::tile_origin(u1 & (T - 1u), d, M), d, pt, LOGNT);
        }
      }
    }
    if (!ok && pt == 0) atomicExch(err, 1);
    pipe::cp_async_drain();
    return;
  }

  // compute group g: local units g, g + 2, ...
  asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kPipeRegsCompute));
  const int g = tid / NT, gt = tid % NT;
  const uint32_t bar = 1u + (uint32_t)g;
  const pipe::SyncNamed sync{bar, (uint32_t)NT};
  for (unsigned i = (unsigned)g; i < nloc; i += 2u) {
    const uint32_t b = i % 3u;
    const bool late = !pipe::mbar_wait(a_full + 8u * b, (i / 3u) & 1u, err);
    if (pipe::group_any(late, bar, NT)) {
      if (gt == 0) atomicExch(err, 1);
      break;
    }
    const unsigned u = blockIdx.x + i * G;
    const unsigned tile = u & (T - 1u);
    // the unit's job pointers: BATCH from its buffer's slot, which stays
    // valid until the buffer is handed back
    const JobPtrs *js = BATCH ? &s_job[b] : jobs;
    const ROpRes *ops = BATCH ? s_op + kPipeBatchOps * b : s_op;
    const uint64_t base = sw2::tile_origin(tile, d, M);
    float up = 0.f, dn = 0.f;
    sw2::run_phases<RB, false, false>(tiles + b * TA, d, s_ph, ops, base, gt, LOGNT, M, js->qdiag, up, dn, sH[g],
                                      sQ[g], &sOut[g], nullptr, sync);
    // run_phases ends with the group's barrier: the tile is finished
    if (!d.has_reduce) {
      if (gt == 0) pipe::mbar_arrive(a_done + 8u * b);
      continue;
    }
    // the tile's partial, summed as reduce_finalize sums a block's; the
    // buffer goes back after the group's barrier below, once every thread
    // has read the job's reduction pointers from its slot
    double2 *const partials = js->partials;
    double pu = (double)up, pv = (double)dn;
    for (int o = 16; o; o >>= 1) {
      pu += __shfl_xor_sync(0xffffffffu, pu, o);
      pv += __shfl_xor_sync(0xffffffffu, pv, o);
    }
    if ((gt & 31) == 0) s_up[g][gt >> 5] = pu, s_dn[g][gt >> 5] = pv;
    sync();
    if (gt == 0) {
      pipe::mbar_arrive(a_done + 8u * b);
      double U = 0.0, D = 0.0;
      for (int w = 0; w < NW; ++w) U += s_up[g][w], D += s_dn[g][w];
      partials[tile] = make_double2(U, D);
    }
  }
  if (BATCH || !d.has_reduce || probe) return;
  if (gt == 0) __threadfence();
  const pipe::SyncNamed both{4u, (uint32_t)(2 * NT)};
  both();

  // one job: the last block to finish combines the tile partials (group 0)
  if (tid == 0) {
    const unsigned t = atomicAdd(jobs[0].ticket, 1u);
    s_last = (t == G - 1u);
  }
  both();
  if (!s_last || tid >= NT) return;
  __threadfence();
  const JobPtrs j0 = jobs[0];
  pipe_finalize<NW>(j0.partials, j0.ticket, j0.step, j0.series, T, tid, err, s_up[0], s_dn[0], sync);
}

// After a batch's reducing pipelined sweep: block j sums job j's T tile
// partials (128 threads, the order of reduce_finalize) and appends its (P,
// norm), NaN when err is set.
__global__ void __launch_bounds__(128) pipe_finalize_kernel(const JobPtrs *__restrict__ jobs, unsigned T,
                                                            const int *err) {
  __shared__ double su[4], sd[4];
  const JobPtrs jp = jobs[blockIdx.x];
  pipe_finalize<4>(jp.partials, jp.ticket, jp.step, jp.series, T, threadIdx.x, err, su, sd, sw2::SyncBlock{});
}

}  // namespace spinrp
