// kernels.cuh -- device code of the random-phase Trotter path (sm_103a).
//
//   init_kernel   : the paper's entangled random-phase state (or its product
//                   state), phases from an in-kernel Philox4x32-10, fused
//                   P(0)/norm reduction.
//   coef_kernel   : FP64 generation of every flip-flop gate's three-shear
//                   coefficients (tan theta/2, sin theta) for dt/2 and dt, and
//                   the FP32 pair closest to a rotation.
//   diag_kernel   : FP64 -> 64-bit fixed-point turn tables of e^{-i tau a_ij/4 s s}.
//   sweep_kernel  : one pass over the whole state in shared-memory tiles of 2^K
//                   amplitudes: applies the pass's gates, the diagonal phase and
//                   the polarization reduction, then writes the tile back.
//   sweep2_kernel : the same pass with register-blocked phases (complex64).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace spinrp {

template <typename R> struct CT;
template <> struct CT<float> { using T = float2; };
template <> struct CT<double> { using T = double2; };

struct LayoutArg {
  uint8_t logical_of[kMaxM];  // physical bit position -> logical spin
};

__device__ __forceinline__ uint64_t deposit_bits(uint64_t v, const uint8_t *pos, int n) {
  uint64_t r = 0;
  for (int k = 0; k < n; ++k) r |= ((v >> k) & 1ull) << pos[k];
  return r;
}

// Insert a zero bit at position b of x.
__device__ __forceinline__ uint32_t insert_zero(uint32_t x, int b) {
  return ((x >> b) << (b + 1)) | (x & ((1u << b) - 1u));
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): 10 rounds of two 32x32
// multiplies (multipliers 0xD2511F53, 0xCD9E8D57) mixed with the counter and a
// key bumped by the Weyl constants 0x9E3779B9, 0xBB67AE85.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

// e^{2 pi i theta / 2^64} for a 64-bit fixed-point turn count theta.
__device__ __forceinline__ double2 cis_turns(uint64_t theta, double) {
  const double turns = (double)(int64_t)theta * 5.421010862427522e-20;  // 2^-64
  double s, c;
  sincospi(2.0 * turns, &s, &c);
  return make_double2(c, s);
}
// FP32 version: split off the nearest quarter turn exactly in integers, take
// sin/cos of the remainder (|r| <= 1/8 turn, so float keeps ~2^-27 turn
// absolute precision) and rotate by the quarter turns.
__device__ __forceinline__ float2 cis_turns(uint64_t theta, float) {
  const int64_t h = (int64_t)(int32_t)(uint32_t)(theta >> 32);  // turns * 2^32, signed
  const int64_t k = (h + (1ll << 29)) >> 30;                     // nearest quarter turn
  const int32_t r = (int32_t)(h - (k << 30));                    // |r| <= 2^29
  float s, c;
  sincospif((float)r * 4.656612873077393e-10f, &s, &c);          // angle = pi * r * 2^-31
  switch ((int)(k & 3)) {
    case 0: return make_float2(c, s);
    case 1: return make_float2(-s, c);
    case 2: return make_float2(-c, -s);
    default: return make_float2(s, -c);
  }
}

template <typename C>
__device__ __forceinline__ C cmul(C a, C b) {
  C r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}

// Deterministic grid reduction of (N_up, N_dn) for the job of this block row:
// block partials in FP64, the last block to finish sums them in block order,
// appends (P, norm) to the job's series at its step counter (slot 0 when
// `reset`) and advances the counter.
__device__ void reduce_finalize(double up, double dn, const JobPtrs &jp, bool reset) {
  double2 *partials = jp.partials;
  unsigned *ticket = jp.ticket;
  __shared__ double s_up[32], s_dn[32];
  __shared__ int s_last;
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
    partials[blockIdx.x] = make_double2(u, d);
    __threadfence();
    const unsigned t = atomicAdd(ticket, 1u);
    s_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double u = 0.0, d = 0.0;
  for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
    const double2 p = __ldcg(&partials[b]);
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
    const int64_t slot = reset ? 0 : *jp.step;
    jp.series[2 * slot] = (U - D) / (U + D);
    jp.series[2 * slot + 1] = U + D;
    *jp.step = slot + 1;
    *ticket = 0u;
  }
}

// ---------------------------------------------------------------------------
// All-site readout (P_{q1}(t) for every spin q).  A reducing sweep leaves per
// block, per tile bit, the weight with that bit up (and the block's norm);
// write_site_partials turns them into per-spin columns and
// sites_finalize_kernel sums the columns over blocks in a fixed order.
// ---------------------------------------------------------------------------
constexpr int kSiteSlots = kMaxK + 1;  // tile bits 0..kMaxK-1, slot kMaxK = norm
constexpr int kMaxWarps = 16;

// Warp-sum v (in the thread's precision) and park it at s_w[warp][slot].
template <typename R>
__device__ __forceinline__ void warp_site_sum(R v, int slot, double *s_w) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) s_w[(threadIdx.x >> 5) * kSiteSlots + slot] = (double)v;
}

// After a __syncthreads that follows every warp_site_sum: block sums over the
// warps in order, written as this block's row of the (M + 1) columns.
__device__ void write_site_partials(const PassDesc d, int M, uint64_t base, const double *s_w,
                                    double *psites) {
  const int nw = (blockDim.x + 31) >> 5, K = d.K;
  const size_t nblk = gridDim.x, blk = blockIdx.x;
  for (int i = threadIdx.x; i <= M; i += blockDim.x) {
    double norm = 0.0;
    for (int w = 0; w < nw; ++w) norm += s_w[w * kSiteSlots + kMaxK];
    double v;
    int col;
    if (i < K) {
      v = 0.0;
      for (int w = 0; w < nw; ++w) v += s_w[w * kSiteSlots + i];
      col = 1 + d.tile_spin[i];
    } else if (i < M) {
      const int o = i - K;
      v = ((base >> d.outer_pos[o]) & 1ull) ? norm : 0.0;
      col = 1 + d.outer_spin[o];
    } else {
      v = norm;
      col = 0;
    }
    psites[col * nblk + blk] = v;
  }
}

// Whole-state scan (after init or load): per block, the norm and the weight
// with each spin up, as the same (M + 1) columns.
template <typename R>
__global__ void __launch_bounds__(256)
state_sites_kernel(const JobPtrs *__restrict__ jobs, int M, LayoutArg lay) {
  const JobPtrs jp = jobs[blockIdx.y];
  const typename CT<R>::T *__restrict__ psi = static_cast<const typename CT<R>::T *>(jp.psi);
  const uint64_t N = 1ull << M;
  R up[kMaxM], norm = 0;
#pragma unroll
  for (int p = 0; p < kMaxM; ++p) up[p] = 0;
  for (uint64_t y = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; y < N;
       y += (uint64_t)gridDim.x * blockDim.x) {
    const typename CT<R>::T v = psi[y];
    const R pr = v.x * v.x + v.y * v.y;
    norm += pr;
#pragma unroll
    for (int p = 0; p < kMaxM; ++p)
      if (p < M && ((y >> p) & 1ull)) up[p] += pr;
  }
  __shared__ double s_w[kMaxWarps * (kMaxM + 1)];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int p = 0; p <= kMaxM; ++p) {
    R v = p < kMaxM ? up[p] : norm;
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) s_w[warp * (kMaxM + 1) + p] = (double)v;
  }
  __syncthreads();
  const size_t nblk = gridDim.x, blk = blockIdx.x;
  for (int i = threadIdx.x; i <= M; i += blockDim.x) {
    const int slot = i < M ? i : kMaxM;
    double v = 0.0;
    for (int w = 0; w < nw; ++w) v += s_w[w * (kMaxM + 1) + slot];
    const int col = i < M ? 1 + lay.logical_of[i] : 0;
    jp.psites[col * nblk + blk] = v;
  }
}

// P of every spin for the entry the preceding reduction recorded (slot
// *step - 1): block q sums columns 0 and 1 + q over the nblk block rows in a
// fixed order, P_q = (2 N_up - N) / N.
__global__ void __launch_bounds__(256)
sites_finalize_kernel(const JobPtrs *__restrict__ jobs, int M, int nblk) {
  const JobPtrs jp = jobs[blockIdx.y];
  const int q = blockIdx.x;
  const double *__restrict__ c0 = jp.psites;
  const double *__restrict__ cq = jp.psites + (size_t)(1 + q) * nblk;
  double n = 0.0, u = 0.0;
  for (int r = threadIdx.x; r < nblk; r += blockDim.x) n += c0[r], u += cq[r];
  __shared__ double sn[256], su[256];
  sn[threadIdx.x] = n;
  su[threadIdx.x] = u;
  __syncthreads();
  for (int h = 128; h; h >>= 1) {
    if (threadIdx.x < h) sn[threadIdx.x] += sn[threadIdx.x + h], su[threadIdx.x] += su[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const int64_t slot = *jp.step - 1;
    jp.site_series[slot * M + q] = (2.0 * su[0] - sn[0]) / sn[0];
  }
}

// ---------------------------------------------------------------------------
// Random-phase initial state.
// ---------------------------------------------------------------------------
// kind INIT_ENTANGLED: an independent phase per basis state of spins 2..M.
// kind INIT_PRODUCT: the paper's product state, spin 1 up and every other spin
// l in (|down> + e^{-i phi_l}|up>)/sqrt 2, phi_l = 2 pi u_l with u_l the top 53
// bits of Philox4x32-10(counter = (l-1, 0, 0, 1), key) times 2^-53; the
// amplitude's phase -sum phi_l over the up spins is summed exactly as 64-bit
// fixed-point turns.
enum InitKind { INIT_ENTANGLED = 0, INIT_PRODUCT = 1 };

// orient: logical mask of the first-colour spins of an oriented state (0 for
// a plain one): amplitudes with an odd number of them up are stored (Im, Re).
template <typename R>
__global__ void __launch_bounds__(256)
init_kernel(const JobPtrs *__restrict__ jobs, int M, LayoutArg lay, uint64_t seed0,
            const uint64_t *__restrict__ seeds, int kind, uint64_t orient) {
  using C = typename CT<R>::T;
  const JobPtrs jp = jobs[blockIdx.y];
  C *__restrict__ psi = static_cast<C *>(jp.psi);
  const uint64_t seed = seeds ? seeds[blockIdx.y] : seed0;
  const uint64_t N = 1ull << M;
  const R amp = (R)exp2(-0.5 * (double)(M - 1));
  const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  // product state: turns u_l * 2^64 of each physical bit position (0 for spin 1)
  __shared__ uint64_t s_turns[kMaxM];
  if (kind == INIT_PRODUCT) {
    for (int p = threadIdx.x; p < M; p += blockDim.x) {
      const int q = lay.logical_of[p];
      uint64_t t = 0;
      if (q > 0) {
        const uint4 w = philox4x32_10(make_uint4((uint32_t)q, 0u, 0u, 1u), key);
        t = ((((uint64_t)w.x << 32) | w.y) >> 11) << 11;
      }
      s_turns[p] = t;
    }
    __syncthreads();
  }
  R up = 0, dn = 0;
  for (uint64_t y = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; y < N;
       y += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t x = 0;
    for (int p = 0; p < M; ++p) x |= ((y >> p) & 1ull) << lay.logical_of[p];
    C v;
    if ((x & 1ull) == 0) {
      v.x = 0, v.y = 0;
    } else if (kind == INIT_PRODUCT) {
      uint64_t th = 0;
      for (int p = 0; p < M; ++p)
        if ((y >> p) & 1ull) th -= s_turns[p];
      const C e = cis_turns(th, (R)0);
      v.x = amp * e.x, v.y = amp * e.y;
      up += v.x * v.x + v.y * v.y;
    } else {
      const uint64_t r = x >> 1;
      const uint4 w = philox4x32_10(make_uint4((uint32_t)r, (uint32_t)(r >> 32), 0u, 0u), key);
      const uint64_t bits = ((uint64_t)w.x << 32) | w.y;
      C e;
      if (sizeof(R) == 8) {
        // u = top 53 bits * 2^-53 exactly as defined; angle 2 pi u
        double s, c;
        sincospi(2.0 * ((double)(bits >> 11) * 1.1102230246251565e-16), &s, &c);
        e.x = (R)c, e.y = (R)s;
      } else {
        const float2 f = cis_turns(bits, 0.0f);
        e.x = (R)f.x, e.y = (R)f.y;
      }
      v.x = amp * e.x, v.y = amp * e.y;
      up += v.x * v.x + v.y * v.y;
    }
    if (__popcll(x & orient) & 1) {
      const R t = v.x;
      v.x = v.y, v.y = t;
    }
    psi[y] = v;
  }
  reduce_finalize((double)up, (double)dn, jp, true);
}

// ---------------------------------------------------------------------------
// Per-evolve FP64 tables.
// ---------------------------------------------------------------------------
__global__ void coef_kernel(const JobPtrs *__restrict__ jobs, int nb, double dt) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= 2 * nb) return;
  const double *__restrict__ bvals = jobs[blockIdx.y].bvals;
  GateCoef *__restrict__ out = const_cast<GateCoef *>(jobs[blockIdx.y].coefs);
  const double tau = (k & 1) ? dt : 0.5 * dt;
  const double th = 0.5 * bvals[k >> 1] * tau;  // exp(-i tau b (SxSx+SySy)) = cos th - i sin th sigma_x
  const double s = sin(th);
  GateCoef g;
  g.s = s;
  g.t = tan(0.5 * th);
  // FP32 shear pair: among +-2 ulps of the rounded values, the one closest to a
  // rotation, |s (1 + t^2) - 2 t| (zero exactly when s = sin 2 atan t)
  const float t0 = (float)g.t, s1 = (float)s;
  float bt = t0, bs2 = s1;
  double best2 = fabs((double)s1 * (1.0 + (double)t0 * t0) - 2.0 * (double)t0);
  for (int dtt = -2; dtt <= 2; ++dtt)
    for (int ds = -2; ds <= 2; ++ds) {
      const float tf = (t0 == 0.0f) ? t0 : __int_as_float(__float_as_int(t0) + dtt);
      const float sf = (s1 == 0.0f) ? s1 : __int_as_float(__float_as_int(s1) + ds);
      const double def = fabs((double)sf * (1.0 + (double)tf * tf) - 2.0 * (double)tf);
      if (def < best2) best2 = def, bt = tf, bs2 = sf;
    }
  g.tf = bt;
  g.sft = bs2;
  out[k] = g;
}

// Per job: the register-blocked program's ops with their FP32 gate
// coefficients looked up once per dt (the sweep kernels copy them as is).
__global__ void resolve_ops_kernel(const JobPtrs *__restrict__ jobs, const ROp *__restrict__ rops,
                                   int nrops) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nrops) return;
  const JobPtrs &jp = jobs[blockIdx.y];
  const ROp r = rops[i];
  ROpRes o;
  o.kind = r.kind, o.combo = r.combo, o.arg = r.arg, o.pad = 0, o.pad2 = 0;
  o.t = 0.f, o.s = 0.f;
  if (r.kind == OP_GATE) {
    const GateCoef g = jp.coefs[r.coef];
    o.t = g.tf, o.s = g.sft;
  }
  jp.sops[i] = o;
}

// q[v][p][p'] (physical positions): turns of the pair phase -tau_v a_ij / 4 (the
// phase of e^{-i tau a_ij s_i s_j} for s_i s_j = +1/4), as 64-bit fixed point.
// tau_0 = dt/2, tau_1 = dt.
__global__ void diag_kernel(const JobPtrs *__restrict__ jobs, LayoutArg lay, int M, double dt) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= 2 * M * M) return;
  const double *__restrict__ a = jobs[blockIdx.y].a;
  uint64_t *__restrict__ q = const_cast<uint64_t *>(jobs[blockIdx.y].qdiag);
  const int v = k / (M * M), p = (k / M) % M, p2 = k % M;
  uint64_t val = 0;
  if (p != p2) {
    const int i = lay.logical_of[p], j = lay.logical_of[p2];
    const double aij = a[(i < j ? i : j) * M + (i < j ? j : i)];
    const double tau = v ? dt : 0.5 * dt;
    const double t = -tau * aij * 0.039788735772973836;  // 1/(8 pi)
    const double f = t - rint(t);                          // [-1/2, 1/2] turns
    val = ((uint64_t)llrint(f * 9.223372036854775808e18)) << 1;
  }
  q[k] = val;
}

// ---------------------------------------------------------------------------
// One sweep.  Each block owns one tile: it loads the tile's 2^K amplitudes
// into shared memory, applies the pass's ops in order and stores the tile.
// ---------------------------------------------------------------------------
// A gate as two real plane rotations: exp(-i theta sigma_x) maps
// (Re a, Im b) and (Re b, Im a) each by [[c, s], [-s, c]], c = cos theta,
// s = sin theta, and each rotation is three shears x += t y, y -= s x,
// x += t y with t = tan(theta/2): three FMAs per plane.  A shear has
// determinant one whatever t and s are rounded to, so rounding leaves no
// uniform gain or loss of norm.
__device__ __forceinline__ void shear_rotate(float2 &a, float2 &b, float t, float s) {
  float x = fmaf(t, b.y, a.x);
  b.y = fmaf(-s, x, b.y);
  a.x = fmaf(t, b.y, x);
  x = fmaf(t, a.y, b.x);
  a.y = fmaf(-s, x, a.y);
  b.x = fmaf(t, a.y, x);
}
__device__ __forceinline__ void shear_rotate(double2 &a, double2 &b, double t, double s) {
  double x = fma(t, b.y, a.x);
  b.y = fma(-s, x, b.y);
  a.x = fma(t, b.y, x);
  x = fma(t, a.y, b.x);
  a.y = fma(-s, x, a.y);
  b.x = fma(t, a.y, x);
}


template <typename R, bool SITES>
__global__ void __launch_bounds__(512)
sweep_kernel(const JobPtrs *__restrict__ jobs, const PassDesc *__restrict__ pdesc,
             const Op *__restrict__ ops, int M) {
  using C = typename CT<R>::T;
  const JobPtrs jp = jobs[blockIdx.y];
  C *__restrict__ psi = static_cast<C *>(jp.psi);
  const GateCoef *__restrict__ coefs = jp.coefs;
  const uint64_t *__restrict__ qdiag = jp.qdiag;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *tile = reinterpret_cast<C *>(smem_raw);
  __shared__ PassDesc d;
  __shared__ uint64_t sH[kMaxK];
  __shared__ uint64_t sQ[kMaxK * kMaxK];
  __shared__ uint64_t sOut;
  __shared__ double s_w[SITES ? kMaxWarps * kSiteSlots : 1];
  {
    const int nwords = (int)(sizeof(PassDesc) / 4);
    for (int w = threadIdx.x; w < nwords; w += blockDim.x)
      reinterpret_cast<int *>(&d)[w] = reinterpret_cast<const int *>(pdesc)[w];
  }
  __syncthreads();
  const int K = d.K;
  const int nt = blockDim.x, tid = threadIdx.x;
  const int lognt = 31 - __clz(nt);
  const int L = lognt < K ? lognt : K;  // tile bits taken from the thread index
  const uint32_t T = 1u << K;
  const uint64_t base = deposit_bits(blockIdx.x, d.outer_pos, M - K);
  const uint64_t off_lo = deposit_bits(tid, d.tile_pos, L);
  auto offset = [&](uint32_t t) -> uint64_t {
    uint64_t o = off_lo;
    for (int q = L; q < K; ++q) o |= (uint64_t)((t >> q) & 1u) << d.tile_pos[q];
    return o;
  };
  for (uint32_t t = tid; t < T; t += nt) tile[t] = psi[base + offset(t)];
  __syncthreads();

  R up = 0, dn = 0;
  for (int k = 0; k < d.nops; ++k) {
    const Op op = ops[d.op0 + k];
    if (op.kind == OP_GATE) {
      const GateCoef g = coefs[op.coef];
      const R c1 = sizeof(R) == 8 ? (R)g.t : (R)g.tf;
      const R s = sizeof(R) == 8 ? (R)g.s : (R)g.sft;
      const int lo = op.u < op.v ? op.u : op.v, hi = op.u < op.v ? op.v : op.u;
      const uint32_t bu = 1u << op.u, bv = 1u << op.v;
      for (uint32_t p = tid; p < (T >> 2); p += nt) {
        const uint32_t t0 = insert_zero(insert_zero(p, lo), hi);
        C a = tile[t0 | bu], b = tile[t0 | bv];
        shear_rotate(a, b, c1, s);
        tile[t0 | bu] = a;
        tile[t0 | bv] = b;
      }
      __syncthreads();
    } else if (op.kind == OP_DIAG) {
      // Theta(x) = sum_{p<p'} q_pp' sigma_p sigma_p' (mod 2^64), split into
      // outer-outer, outer-tile and tile-tile parts.
      const uint64_t *q = qdiag + (size_t)op.arg * M * M;
      const int nout = M - K;
      if (tid < K) {
        const int p = d.tile_pos[tid];
        uint64_t h = 0;
        for (int o = 0; o < nout; ++o) {
          const int po = d.outer_pos[o];
          const uint64_t v = q[p * M + po];
          h += ((base >> po) & 1ull) ? v : (0ull - v);
        }
        sH[tid] = h;
      } else if (tid == K) {
        uint64_t s = 0;
        for (int o = 0; o < nout; ++o)
          for (int o2 = o + 1; o2 < nout; ++o2) {
            const int p = d.outer_pos[o], p2 = d.outer_pos[o2];
            const uint64_t v = q[p * M + p2];
            s += (((base >> p) ^ (base >> p2)) & 1ull) ? (0ull - v) : v;
          }
        sOut = s;
      }
      for (int w = tid; w < K * K; w += nt) {
        const int a = w / K, b = w % K;
        sQ[w] = q[d.tile_pos[a] * M + d.tile_pos[b]];
      }
      __syncthreads();
      // per-thread part: tile bits 0..L-1 come from tid
      uint64_t thr = sOut;
      for (int a = 0; a < L; ++a) {
        const uint64_t ba = (tid >> a) & 1u;
        thr += ba ? sH[a] : (0ull - sH[a]);
        for (int b = a + 1; b < L; ++b)
          thr += (ba ^ ((tid >> b) & 1u)) ? (0ull - sQ[a * K + b]) : sQ[a * K + b];
      }
      for (uint32_t t = tid; t < T; t += nt) {
        uint64_t th = thr;
        for (int a = L; a < K; ++a) {
          const uint32_t ba = (t >> a) & 1u;
          uint64_t f = sH[a];
          for (int b = 0; b < L; ++b)
            f += ((tid >> b) & 1u) ? sQ[b * K + a] : (0ull - sQ[b * K + a]);
          th += ba ? f : (0ull - f);
          for (int b = a + 1; b < K; ++b)
            th += (ba ^ ((t >> b) & 1u)) ? (0ull - sQ[a * K + b]) : sQ[a * K + b];
        }
        const C e = cis_turns(th, (R)0);
        tile[t] = cmul(tile[t], e);
      }
      __syncthreads();
    } else if (op.kind == OP_REDUCE) {
      R tsum = 0, uhi[kMaxK];
#pragma unroll
      for (int q = 0; q < kMaxK; ++q) uhi[q] = 0;
      for (uint32_t t = tid; t < T; t += nt) {
        const C a = tile[t];
        const R pr = a.x * a.x + a.y * a.y;
        const uint64_t bit = d.site_tile >= 0 ? ((t >> d.site_tile) & 1u)
                                              : ((base >> d.site_pos) & 1ull);
        if (bit) up += pr;
        else dn += pr;
        if constexpr (SITES) {
          tsum += pr;
#pragma unroll
          for (int q = 0; q < kMaxK; ++q)
            if (q >= L && q < K && ((t >> q) & 1u)) uhi[q] += pr;
        }
      }
      if constexpr (SITES) {
        // tile bits below L come from the thread index: the thread's whole sum
#pragma unroll
        for (int q = 0; q < kMaxK; ++q)
          warp_site_sum<R>(q < L ? (((tid >> q) & 1) ? tsum : (R)0) : uhi[q], q, s_w);
        warp_site_sum<R>(tsum, kMaxK, s_w);
      }
      __syncthreads();  // later ops overwrite the tile
    }
  }
  if (!d.relabel) {
    for (uint32_t t = tid; t < T; t += nt) psi[base + offset(t)] = tile[t];
  } else {
    // output tile bit q holds the spin that input tile bit perm[q] held
    for (uint32_t t = tid; t < T; t += nt) {
      uint32_t ti = 0;
      for (int q = 0; q < K; ++q) ti |= ((t >> q) & 1u) << d.perm[q];
      psi[base + offset(t)] = tile[ti];
    }
  }
  if constexpr (SITES)
    if (d.has_reduce) write_site_partials(d, M, base, s_w, jp.psites);
  if (d.has_reduce) reduce_finalize((double)up, (double)dn, jp, false);
}

// Gather amplitudes at physical indices into a staging buffer (FP64 pairs).
// orient: physical positions of the first-colour spins of an oriented state
// (0 for a plain one); those amplitudes stored (Im, Re) are read back as (Re, Im).
template <typename R>
__global__ void gather_kernel(const typename CT<R>::T *__restrict__ psi,
                              const int64_t *__restrict__ idx, int64_t n, double2 *out, uint64_t orient) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const typename CT<R>::T v = psi[idx[k]];
    const bool sw = __popcll((uint64_t)idx[k] & orient) & 1;
    out[k] = sw ? make_double2((double)v.y, (double)v.x) : make_double2((double)v.x, (double)v.y);
  }
}

template <typename R>
__global__ void scatter_kernel(typename CT<R>::T *__restrict__ psi, const int64_t *__restrict__ idx,
                               int64_t n, const double2 *__restrict__ in, uint64_t orient) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    typename CT<R>::T v;
    const bool sw = __popcll((uint64_t)idx[k] & orient) & 1;
    v.x = (R)(sw ? in[k].y : in[k].x);
    v.y = (R)(sw ? in[k].x : in[k].y);
    psi[idx[k]] = v;
  }
}

// Polarization/norm of the whole state (after a load).
template <typename R>
__global__ void __launch_bounds__(256)
observe_kernel(const JobPtrs *__restrict__ jobs, int M, int site_pos) {
  const JobPtrs jp = jobs[blockIdx.y];
  const typename CT<R>::T *__restrict__ psi = static_cast<const typename CT<R>::T *>(jp.psi);
  const uint64_t N = 1ull << M;
  double up = 0, dn = 0;
  for (uint64_t y = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; y < N;
       y += (uint64_t)gridDim.x * blockDim.x) {
    const typename CT<R>::T v = psi[y];
    const double pr = (double)v.x * v.x + (double)v.y * v.y;
    if ((y >> site_pos) & 1ull) up += pr;
    else dn += pr;
  }
  reduce_finalize(up, dn, jp, true);
}

// ===========================================================================
// Register-blocked sweep (complex64).  The tile lives in shared memory with
// an XOR swizzle; global<->shared copies are 16-byte cp.async loads and
// 16-byte stores; between them the pass runs as a sequence of phases, each a
// register-resident 32-amplitude subcube per thread (see PhaseDesc).
// ===========================================================================
namespace sw2 {

// Shared-memory slot of tile index t: the low four bits are XORed with bits
// 4-7, 8-11 and 12-15.  Linear over XOR, so slot(a ^ b) = slot(a) ^ slot(b);
// lanes that differ in four tile bits of distinct residues mod 4 hit 16
// distinct 8-byte bank pairs.
__device__ __forceinline__ uint32_t slot(uint32_t t) {
  return t ^ (((t >> 4) ^ (t >> 8) ^ (t >> 12)) & 15u);
}

// Packed FP32x2 arithmetic on 64-bit registers (two lanes per instruction,
// sm_100 and later).  A pack holds (low lane, high lane) = (bit clear, bit set).
typedef unsigned long long u64;
__device__ __forceinline__ u64 mul2(u64 a, u64 b) {
  u64 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ u64 add2(u64 a, u64 b) {
  u64 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ u64 fma2(u64 a, u64 b, u64 c) {
  u64 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ u64 pack2(float lo, float hi) {
  u64 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ float2 unpack2(u64 v) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
  return r;
}

// A thread's 2^RB amplitudes in a phase are NP = 2^(RB-1) packs: RE[j] =
// (re with register bit 0 clear, re with it set), IM[j] likewise, j = register
// bits 1..RB-1.  Register bit 0 (the "pack bit") is chosen by the host as the
// bit with the fewest gates in the phase.

// In-place x += a * b on packed FP32x2 (the accumulator keeps its register,
// so a gate leaves every pack where it found it).
__device__ __forceinline__ void fma2_acc(u64 &x, u64 a, u64 b) {
  asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(x) : "l"(a), "l"(b));
}

// Three in-place shears on the plane (high lane of P, low lane of Q) or
// (low lane of P, high lane of Q): X += t Y, Y += n X, X += t Y.
__device__ __forceinline__ void shear_hi_lo(u64 &P, u64 &Q, float t, float n) {
  asm("{\n\t.reg .f32 pl, ph, ql, qh;\n\t"
      "mov.b64 {pl, ph}, %0;\n\tmov.b64 {ql, qh}, %1;\n\t"
      "fma.rn.f32 ph, %2, ql, ph;\n\tfma.rn.f32 ql, %3, ph, ql;\n\tfma.rn.f32 ph, %2, ql, ph;\n\t"
      "mov.b64 %0, {pl, ph};\n\tmov.b64 %1, {ql, qh};\n\t}"
      : "+l"(P), "+l"(Q) : "f"(t), "f"(n));
}
__device__ __forceinline__ void shear_lo_hi(u64 &P, u64 &Q, float t, float n) {
  asm("{\n\t.reg .f32 pl, ph, ql, qh;\n\t"
      "mov.b64 {pl, ph}, %0;\n\tmov.b64 {ql, qh}, %1;\n\t"
      "fma.rn.f32 pl, %2, qh, pl;\n\tfma.rn.f32 qh, %3, pl, qh;\n\tfma.rn.f32 pl, %2, qh, pl;\n\t"
      "mov.b64 %0, {pl, ph};\n\tmov.b64 %1, {ql, qh};\n\t}"
      : "+l"(P), "+l"(Q) : "f"(t), "f"(n));
}

// Gate on register bits (JU + 1, JV + 1): two amplitude pairs per packed
// instruction, same three-shear update as shear_rotate, in place.
template <int NP, int JU, int JV>
__device__ __forceinline__ void gate_packed(u64 (&RE)[NP], u64 (&IM)[NP], float t, float s) {
  const u64 t2 = pack2(t, t), n2 = pack2(-s, -s);
  // plane (Re a, Im b) = (RE[j], IM[k]); plane (Re b, Im a) = (RE[k], IM[j]);
  // each shear step over every plane of the gate before the next (independent
  // instructions back to back)
#pragma unroll
  for (int j = 0; j < NP; ++j)
    if (((j >> JU) & 1) == 1 && ((j >> JV) & 1) == 0) {
      const int k = j ^ (1 << JU) ^ (1 << JV);
      fma2_acc(RE[j], t2, IM[k]);
      fma2_acc(RE[k], t2, IM[j]);
    }
#pragma unroll
  for (int j = 0; j < NP; ++j)
    if (((j >> JU) & 1) == 1 && ((j >> JV) & 1) == 0) {
      const int k = j ^ (1 << JU) ^ (1 << JV);
      fma2_acc(IM[k], n2, RE[j]);
      fma2_acc(IM[j], n2, RE[k]);
    }
#pragma unroll
  for (int j = 0; j < NP; ++j)
    if (((j >> JU) & 1) == 1 && ((j >> JV) & 1) == 0) {
      const int k = j ^ (1 << JU) ^ (1 << JV);
      fma2_acc(RE[j], t2, IM[k]);
      fma2_acc(RE[k], t2, IM[j]);
    }
}

// Gate on the pack bit and register bit JV + 1: the pair is the high lane of
// pack j (JV clear) and the low lane of pack j + 2^JV; scalar arithmetic.
template <int NP, int JV>
__device__ __forceinline__ void gate_packbit(u64 (&RE)[NP], u64 (&IM)[NP], float t, float s) {
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    if (((j >> JV) & 1) == 0) {
      const int k = j | (1 << JV);
      // a = high lanes of pack j, b = low lanes of pack k:
      // plane (Re a, Im b) = (RE[j].hi, IM[k].lo); plane (Re b, Im a) = (RE[k].lo, IM[j].hi)
      shear_hi_lo(RE[j], IM[k], t, -s);
      shear_lo_hi(RE[k], IM[j], t, -s);
    }
  }
}

// combo = index of (ku < kv) among the RB(RB-1)/2 register-bit pairs in
// lexicographic order: the first RB-1 pair the pack bit (ku = 0).
__device__ __forceinline__ void gate_combo(u64 (&RE)[16], u64 (&IM)[16], int combo, float t, float s) {
  switch (combo) {
    case 0: gate_packbit<16, 0>(RE, IM, t, s); break;
    case 1: gate_packbit<16, 1>(RE, IM, t, s); break;
    case 2: gate_packbit<16, 2>(RE, IM, t, s); break;
    case 3: gate_packbit<16, 3>(RE, IM, t, s); break;
    case 4: gate_packed<16, 0, 1>(RE, IM, t, s); break;
    case 5: gate_packed<16, 0, 2>(RE, IM, t, s); break;
    case 6: gate_packed<16, 0, 3>(RE, IM, t, s); break;
    case 7: gate_packed<16, 1, 2>(RE, IM, t, s); break;
    case 8: gate_packed<16, 1, 3>(RE, IM, t, s); break;
    default: gate_packed<16, 2, 3>(RE, IM, t, s); break;
  }
}
__device__ __forceinline__ void gate_combo(u64 (&RE)[32], u64 (&IM)[32], int combo, float t, float s) {
  switch (combo) {
    case 0: gate_packbit<32, 0>(RE, IM, t, s); break;
    case 1: gate_packbit<32, 1>(RE, IM, t, s); break;
    case 2: gate_packbit<32, 2>(RE, IM, t, s); break;
    case 3: gate_packbit<32, 3>(RE, IM, t, s); break;
    case 4: gate_packbit<32, 4>(RE, IM, t, s); break;
    case 5: gate_packed<32, 0, 1>(RE, IM, t, s); break;
    case 6: gate_packed<32, 0, 2>(RE, IM, t, s); break;
    case 7: gate_packed<32, 0, 3>(RE, IM, t, s); break;
    case 8: gate_packed<32, 0, 4>(RE, IM, t, s); break;
    case 9: gate_packed<32, 1, 2>(RE, IM, t, s); break;
    case 10: gate_packed<32, 1, 3>(RE, IM, t, s); break;
    case 11: gate_packed<32, 1, 4>(RE, IM, t, s); break;
    case 12: gate_packed<32, 2, 3>(RE, IM, t, s); break;
    case 13: gate_packed<32, 2, 4>(RE, IM, t, s); break;
    default: gate_packed<32, 3, 4>(RE, IM, t, s); break;
  }
}

// lowest set bit of a compile-time g in 1..31 (Gray-code walk)
__host__ __device__ constexpr int ctz5(int g) {
  return (g & 1) ? 0 : (g & 2) ? 1 : (g & 4) ? 2 : (g & 8) ? 3 : 4;
}
// same for g in 1..63; gray(g) = g ^ (g >> 1) differs from gray(g - 1) in bit
// ctz6(g), which gray(g) has set when gray_up(g)
__host__ __device__ constexpr int ctz6(int g) { return (g & 31) ? ctz5(g & 31) : 5; }
__host__ __device__ constexpr bool gray_up(int g) { return (((g ^ (g >> 1)) >> ctz6(g)) & 1) != 0; }

// 8-byte asynchronous global->shared copy (one amplitude): the swizzle may
// move an amplitude pair to an odd slot, so 16-byte copies would misalign.
__device__ __forceinline__ void cp_async8(uint32_t smem_addr, const void *gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_addr), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(uint32_t smem_addr, const void *gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_addr), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(uint32_t smem_addr, const void *gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}


// Barrier of the threads a tile's phases run on (the whole block).
struct SyncBlock {
  __device__ __forceinline__ void operator()() const { __syncthreads(); }
};

// Origin of tile `blk` of a pass: lane k places bit k of the tile index at
// outer_pos[k] (M - K < 32 outer bits), a warp OR-reduction assembles the
// offset.  Called by whole warps.
__device__ __forceinline__ uint64_t tile_origin(unsigned blk, const PassDesc &d, int M) {
  const int lane = threadIdx.x & 31;
  const uint64_t c = lane < M - d.K ? (uint64_t)((blk >> lane) & 1u) << d.outer_pos[lane] : 0ull;
  const uint32_t lo = __reduce_or_sync(0xffffffffu, (uint32_t)c);
  const uint32_t hi = __reduce_or_sync(0xffffffffu, (uint32_t)(c >> 32));
  return ((uint64_t)hi << 32) | lo;
}

// Global -> shared copy of a tile by the 2^lognt threads tid of its group
// (8-byte async copies; 16 consecutive threads read one 128-byte run).
// Input amplitude a = tid + nt * e: tile bits 0..lognt-1 from tid, the RB high
// bits from e, e walked in Gray-code order in runs of eight: each copy moves
// the source by +-2^tile_pos (a compile-time sign) and the destination slot by
// one XOR (the slot is XOR-linear); each run starts afresh from the thread's
// origin, so the address chains stay short.
template <int RB>
__device__ __forceinline__ void load_tile(const float2 *psi, uint64_t base, const PassDesc &d, int tid,
                                          int lognt, uint32_t sbase) {
  constexpr int NA = 1 << RB;
  uint64_t off_amp_lo = 0;
  for (int k = 0; k < lognt; ++k)
    if ((tid >> k) & 1) off_amp_lo |= 1ull << d.tile_pos[k];
  int64_t dg[RB];
  uint32_t ds[RB];
#pragma unroll
  for (int k = 0; k < RB; ++k) {
    dg[k] = (int64_t)8 << d.tile_pos[lognt + k];
    ds[k] = slot(1u << (lognt + k)) << 3;
  }
  const char *src0 = reinterpret_cast<const char *>(psi + base + off_amp_lo);
  const uint32_t sb0 = slot((uint32_t)tid) << 3;
  const char *src = src0;
  uint32_t sb = sb0;
#pragma unroll
  for (int g = 0; g < NA; ++g) {
    if ((g & 7) == 0) {
      src = src0, sb = sb0;
#pragma unroll
      for (int k = 0; k < RB; ++k)
        if (((g ^ (g >> 1)) >> k) & 1) src += dg[k], sb ^= ds[k];
    } else {
      const int k = ctz6(g);
      src += gray_up(g) ? dg[k] : -dg[k];
      sb ^= ds[k];
    }
    cp_async8(sbase + sb, src);
  }
}

// L2 prefetch of the tile at origin base2: one 128-byte run (tile bits 0..3,
// the low physical bits) per request; run r = tid + nt * i (tile bits 4.. of
// its first amplitude): bits from tid once, then the RB - 4 high bits per run.
template <int RB>
__device__ __forceinline__ void prefetch_tile(const float2 *psi, uint64_t base2, const PassDesc &d, int tid,
                                              int lognt) {
  uint64_t ot = base2;
  for (int b = 0; b < lognt; ++b)
    if ((tid >> b) & 1) ot |= 1ull << d.tile_pos[4 + b];
#pragma unroll
  for (int i = 0; i < (1 << (RB - 4)); ++i) {
    uint64_t off = ot;
#pragma unroll
    for (int b = 0; b < RB - 4; ++b)
      if ((i >> b) & 1) off |= 1ull << d.tile_pos[4 + lognt + b];
    asm volatile("prefetch.global.L2 [%0];" ::"l"(psi + off));
  }
}

// Tile index of this thread's subcube origin in phase ph (register bits clear).
__device__ __forceinline__ uint32_t thread_origin(const PhaseDesc &ph, int tid, int lognt) {
  uint32_t t0 = 0;
  for (int k = 0; k < 5; ++k) t0 |= ((uint32_t)(tid >> k) & 1u) << ph.lanes[k];
  for (int k = 0; k < lognt - 5; ++k) t0 |= ((uint32_t)(tid >> (5 + k)) & 1u) << ph.warps[k];
  return t0;
}

// The diagonal phase e^{-i tau D}, amplitude by amplitude in shared memory.
// ORIENT: amplitudes of odd orientation are stored (Im, Re) and take the
// conjugate phase (the stored word is i conj(psi), and i conj(psi e^{ia}) =
// i conj(psi) e^{-ia}).  Kept out of line: only systems with S^zS^z terms run
// it, and the sweep's gate code stays smaller (measured 2 % faster on
// dipolar stars, unchanged on XY ladders).
template <int RB, bool ORIENT, typename Sync>
__device__ __noinline__ void diag_phase(float2 *tile2, const PassDesc &d, const PhaseDesc &ph,
                                           const ROpRes &op, uint64_t base, int tid, int lognt, int M,
                                           const uint64_t *__restrict__ qdiag, uint64_t *sH, uint64_t *sQ,
                                           uint64_t *sOut, uint32_t s0, const uint32_t (&sm)[RB], Sync sync) {
  constexpr int NA = 1 << RB;
  const int K = d.K, nt = 1 << lognt;
  const int nout = M - K;
  // Theta(x) = sum_{p<p'} q_pp' sigma_p sigma_p' (mod 2^64) split into
  // outer-outer (sOut), outer-tile (sH) and tile-tile (sQ) parts
  uint32_t t0 = 0;
  for (int k = 0; k < 5; ++k) t0 |= ((uint32_t)(tid >> k) & 1u) << ph.lanes[k];
  for (int k = 0; k < lognt - 5; ++k) t0 |= ((uint32_t)(tid >> (5 + k)) & 1u) << ph.warps[k];
  const uint64_t *q = qdiag + (size_t)op.arg * M * M;
  if (tid < K) {
    const int pp = d.tile_pos[tid];
    uint64_t h = 0;
    for (int o = 0; o < nout; ++o) {
      const int po = d.outer_pos[o];
      const uint64_t v = q[pp * M + po];
      h += ((base >> po) & 1ull) ? v : (0ull - v);
    }
    sH[tid] = h;
  } else if (tid == K) {
    uint64_t s = 0;
    for (int o = 0; o < nout; ++o)
      for (int o2 = o + 1; o2 < nout; ++o2) {
        const int pa = d.outer_pos[o], pb = d.outer_pos[o2];
        const uint64_t v = q[pa * M + pb];
        s += (((base >> pa) ^ (base >> pb)) & 1ull) ? (0ull - v) : v;
      }
    *sOut = s;
  }
  for (int w = tid; w < K * K; w += nt) sQ[w] = q[d.tile_pos[w / K] * M + d.tile_pos[w % K]];
  sync();
  uint32_t isreg = 0;
  for (int k = 0; k < RB; ++k) isreg |= 1u << ph.rb[k];
  // fixed part (tile bits from the thread index) once per thread
  uint64_t th0 = *sOut;
  for (int x = 0; x < K; ++x) {
    if ((isreg >> x) & 1u) continue;
    const uint32_t bx = (t0 >> x) & 1u;
    th0 += bx ? sH[x] : (0ull - sH[x]);
    for (int y = x + 1; y < K; ++y) {
      if ((isreg >> y) & 1u) continue;
      th0 += (bx ^ ((t0 >> y) & 1u)) ? (0ull - sQ[x * K + y]) : sQ[x * K + y];
    }
  }
  // field on each register bit from the fixed bits, once per thread
  uint64_t G[RB];
#pragma unroll
  for (int k = 0; k < RB; ++k) {
    const int rk = ph.rb[k];
    uint64_t g = sH[rk];
    for (int x = 0; x < K; ++x) {
      if ((isreg >> x) & 1u) continue;
      g += ((t0 >> x) & 1u) ? sQ[x * K + rk] : (0ull - sQ[x * K + rk]);
    }
    G[k] = g;
  }
  // the register combinations in Gray-code order: with sigma_k = +1 for a
  // set bit and -1 for a clear one, Theta = th0 + sum_k sigma_k G_k +
  // sum_{k<l} sigma_k sigma_l Q_kl; flipping bit k changes Theta by
  // -2 sigma_k F_k, F_k = G_k + sum_{l!=k} sigma_l Q_kl its field, and
  // every other field F_l by -2 sigma_k Q_kl (exact, modulo 2^64)
  uint64_t Qr[RB][RB], F[RB];
#pragma unroll
  for (int k = 0; k < RB; ++k)
#pragma unroll
    for (int l = 0; l < RB; ++l)
      Qr[k][l] = k == l ? 0ull : sQ[ph.rb[k < l ? k : l] * K + ph.rb[k < l ? l : k]];
  uint64_t th = th0;
#pragma unroll
  for (int k = 0; k < RB; ++k) {
    th -= G[k];
    F[k] = G[k];
#pragma unroll
    for (int l = 0; l < RB; ++l) {
      if (l == k) continue;
      F[k] -= Qr[k][l];
      if (l > k) th += Qr[k][l];
    }
  }
  uint32_t s = s0;
  // orientation of the current amplitude and of each register bit
  uint32_t ori = 0, obit[RB];
  if constexpr (ORIENT) {
    ori = (__popc(t0 & d.black_tile) ^ __popcll(base & d.black_outer)) & 1u;
#pragma unroll
    for (int k = 0; k < RB; ++k) obit[k] = (d.black_tile >> ph.rb[k]) & 1u;
  }
#pragma unroll
  for (int g = 0; g < NA; ++g) {
    if (g) {
      const int k = ctz6(g);
      // sigma_k before the flip: +1 when the bit is set in gray(g - 1)
      const bool was_up = ((((g - 1) ^ ((g - 1) >> 1)) >> k) & 1) != 0;
      th += was_up ? (0ull - 2ull * F[k]) : 2ull * F[k];
#pragma unroll
      for (int l = 0; l < RB; ++l)
        if (l != k) F[l] += was_up ? (0ull - 2ull * Qr[l][k]) : 2ull * Qr[l][k];
      s ^= sm[k];
      if constexpr (ORIENT) ori ^= obit[k];
    }
    float2 e = cis_turns(th, 0.0f);
    if constexpr (ORIENT) e.y = ori ? -e.y : e.y;
    tile2[s] = cmul(tile2[s], e);
  }
  sync();
}

// Register-blocked phases of an oriented program (see Orientation): the
// thread's 2^RB amplitudes are NA words P[j], j = register bits (the first NB
// = ph.nb of them of the first colour), each the stored (Re, Im) or (Im, Re)
// pair as is.  A gate on register bits (JU < NB <= JV) updates the pairs (j, k = j ^
// 2^JU ^ 2^JV), j with bit JU set, by P[j] += T P[k]; P[k] += S P[j]; P[j] +=
// T P[k] (packed FP32x2), with T = (t, -t), S = (-s, s) when amplitude j is
// stored (Re, Im) and both negated when it is stored (Im, Re): the three
// shears of shear_rotate, the second plane's written y-first (y -= t x,
// x += s y, y -= t x, the same rotation).  Orientation of j = parity of its
// first-colour register bits (compile time) XOR the thread's (folded into T, S).
// parity of the low nb bits of j (folded to a constant for a constant j)
__device__ __forceinline__ bool par_low(int j, int nb) { return (__popc((unsigned)j & ((1u << nb) - 1u)) & 1) != 0; }

template <int NA, int NB, int JU, int JV>
__device__ __forceinline__ void gate_oriented(u64 (&P)[NA], u64 T, u64 S) {
  constexpr u64 kNeg = 0x8000000080000000ull;
  const u64 Tn = T ^ kNeg, Sn = S ^ kNeg;
#pragma unroll
  for (int j = 0; j < NA; ++j)
    if (((j >> JU) & 1) == 1 && ((j >> JV) & 1) == 0)
      fma2_acc(P[j], par_low(j, NB) ? Tn : T, P[j ^ (1 << JU) ^ (1 << JV)]);
#pragma unroll
  for (int j = 0; j < NA; ++j)
    if (((j >> JU) & 1) == 1 && ((j >> JV) & 1) == 0)
      fma2_acc(P[j ^ (1 << JU) ^ (1 << JV)], par_low(j, NB) ? Sn : S, P[j]);
#pragma unroll
  for (int j = 0; j < NA; ++j)
    if (((j >> JU) & 1) == 1 && ((j >> JV) & 1) == 0)
      fma2_acc(P[j], par_low(j, NB) ? Tn : T, P[j ^ (1 << JU) ^ (1 << JV)]);
}

// Gate on register bits (ku, kv) of a phase with nb first-colour register
// bits: key = 64 nb + 8 ku + kv.
__device__ __forceinline__ void gate_combo_oriented(u64 (&P)[64], int key, u64 T, u64 S) {
  switch (key) {
    case 130: gate_oriented<64, 2, 0, 2>(P, T, S); break;
    case 131: gate_oriented<64, 2, 0, 3>(P, T, S); break;
    case 132: gate_oriented<64, 2, 0, 4>(P, T, S); break;
    case 133: gate_oriented<64, 2, 0, 5>(P, T, S); break;
    case 138: gate_oriented<64, 2, 1, 2>(P, T, S); break;
    case 139: gate_oriented<64, 2, 1, 3>(P, T, S); break;
    case 140: gate_oriented<64, 2, 1, 4>(P, T, S); break;
    case 141: gate_oriented<64, 2, 1, 5>(P, T, S); break;
    case 195: gate_oriented<64, 3, 0, 3>(P, T, S); break;
    case 196: gate_oriented<64, 3, 0, 4>(P, T, S); break;
    case 197: gate_oriented<64, 3, 0, 5>(P, T, S); break;
    case 203: gate_oriented<64, 3, 1, 3>(P, T, S); break;
    case 204: gate_oriented<64, 3, 1, 4>(P, T, S); break;
    case 205: gate_oriented<64, 3, 1, 5>(P, T, S); break;
    case 211: gate_oriented<64, 3, 2, 3>(P, T, S); break;
    case 212: gate_oriented<64, 3, 2, 4>(P, T, S); break;
    case 213: gate_oriented<64, 3, 2, 5>(P, T, S); break;
    case 260: gate_oriented<64, 4, 0, 4>(P, T, S); break;
    case 261: gate_oriented<64, 4, 0, 5>(P, T, S); break;
    case 268: gate_oriented<64, 4, 1, 4>(P, T, S); break;
    case 269: gate_oriented<64, 4, 1, 5>(P, T, S); break;
    case 276: gate_oriented<64, 4, 2, 4>(P, T, S); break;
    case 277: gate_oriented<64, 4, 2, 5>(P, T, S); break;
    case 284: gate_oriented<64, 4, 3, 4>(P, T, S); break;
    case 285: gate_oriented<64, 4, 3, 5>(P, T, S); break;
    default: break;
  }
}
__device__ __forceinline__ void gate_combo_oriented(u64 (&P)[32], int key, u64 T, u64 S) {
  switch (key) {
    case 130: gate_oriented<32, 2, 0, 2>(P, T, S); break;
    case 131: gate_oriented<32, 2, 0, 3>(P, T, S); break;
    case 132: gate_oriented<32, 2, 0, 4>(P, T, S); break;
    case 138: gate_oriented<32, 2, 1, 2>(P, T, S); break;
    case 139: gate_oriented<32, 2, 1, 3>(P, T, S); break;
    case 140: gate_oriented<32, 2, 1, 4>(P, T, S); break;
    case 195: gate_oriented<32, 3, 0, 3>(P, T, S); break;
    case 196: gate_oriented<32, 3, 0, 4>(P, T, S); break;
    case 203: gate_oriented<32, 3, 1, 3>(P, T, S); break;
    case 204: gate_oriented<32, 3, 1, 4>(P, T, S); break;
    case 211: gate_oriented<32, 3, 2, 3>(P, T, S); break;
    case 212: gate_oriented<32, 3, 2, 4>(P, T, S); break;
    default: break;
  }
}

template <int RB, bool SITES>
__device__ __forceinline__ void oriented_phase(float2 *tile2, const PassDesc &d, const PhaseDesc &ph,
                                               const ROpRes *ops, uint64_t base, int tid, int lognt,
                                               float &up, float &dn, double *s_w, uint32_t s0,
                                               const uint32_t (&sm)[RB], uint32_t outer_par) {
  constexpr int NA = 1 << RB;
  const uint32_t t0 = thread_origin(ph, tid, lognt);
  const int key0 = 64 * ph.nb;
  // the thread's orientation: its fixed tile bits and the tile's outer bits
  const uint32_t tp = (__popc(t0 & d.black_tile) & 1u) ^ outer_par;
  const u64 flip = tp ? 0x8000000080000000ull : 0ull;
  u64 P[NA];
  const char *tb = reinterpret_cast<const char *>(tile2);
  uint32_t mb[RB];
#pragma unroll
  for (int k = 0; k < RB; ++k) mb[k] = sm[k] << 3;
  const uint32_t ob = s0 << 3;
  {
    uint32_t o = ob;
#pragma unroll
    for (int g = 0; g < NA; ++g) {
      const int j = g ^ (g >> 1);
      if ((g & 7) == 0) {
        o = ob;
#pragma unroll
        for (int k = 0; k < RB; ++k)
          if ((j >> k) & 1) o ^= mb[k];
      } else {
        o ^= mb[ctz6(g)];
      }
      P[j] = *reinterpret_cast<const u64 *>(tb + o);
    }
  }
  ROpRes cur = ops[0];
  for (int k = 0; k < ph.nops; ++k) {
    const ROpRes nxt = ops[k + 1 < ph.nops ? k + 1 : k];  // prefetch
    if (cur.kind == OP_GATE) {
      const u64 T = pack2(cur.t, -cur.t) ^ flip, S = pack2(-cur.s, cur.s) ^ flip;
      gate_combo_oriented(P, key0 + cur.combo, T, S);
    } else if (cur.kind == OP_REDUCE) {
      int kr = -1;
#pragma unroll
      for (int q = 0; q < RB; ++q)
        if (ph.rb[q] == d.site_tile) kr = q;
      const uint32_t fixed_bit = d.site_tile < 0 ? (uint32_t)((base >> d.site_pos) & 1ull)
                                                 : (t0 >> d.site_tile) & 1u;
      float tsum = 0.f, ureg[RB];
#pragma unroll
      for (int q = 0; q < RB; ++q) ureg[q] = 0.f;
#pragma unroll
      for (int j = 0; j < NA; ++j) {
        const float2 v = unpack2(P[j]);
        const float pr = fmaf(v.x, v.x, v.y * v.y);
        const uint32_t bit = kr >= 0 ? ((uint32_t)(j >> kr) & 1u) : fixed_bit;
        if (bit) up += pr;
        else dn += pr;
        if constexpr (SITES) {
          tsum += pr;
#pragma unroll
          for (int q = 0; q < RB; ++q)
            if ((j >> q) & 1) ureg[q] += pr;
        }
      }
      if constexpr (SITES) {
#pragma unroll
        for (int q = 0; q < kMaxK; ++q) {
          float v = ((t0 >> q) & 1u) ? tsum : 0.f;
#pragma unroll
          for (int k2 = 0; k2 < RB; ++k2)
            if (ph.rb[k2] == q) v = ureg[k2];
          warp_site_sum<float>(v, q, s_w);
        }
        warp_site_sum<float>(tsum, kMaxK, s_w);
      }
    }
    cur = nxt;
  }
  {
    char *tw = reinterpret_cast<char *>(tile2);
    uint32_t o = ob;
#pragma unroll
    for (int g = 0; g < NA; ++g) {
      const int j = g ^ (g >> 1);
      if ((g & 7) == 0) {
        o = ob;
#pragma unroll
        for (int k = 0; k < RB; ++k)
          if ((j >> k) & 1) o ^= mb[k];
      } else {
        o ^= mb[ctz6(g)];
      }
      *reinterpret_cast<u64 *>(tw + o) = P[j];
    }
  }
}

// The pass's phases on one tile in shared memory, run by the 2^lognt threads
// tid of its group; `sync` is the group's barrier, sH/sQ/sOut the group's
// diagonal-phase scratch, s_w the all-site scratch (SITES only).  ORIENT: the
// program and the state are oriented (see Orientation).
template <int RB, bool SITES, bool ORIENT, typename Sync>
__device__ __forceinline__ void run_phases(float2 *tile2, const PassDesc &d, const PhaseDesc *s_ph,
                                           const ROpRes *s_op, uint64_t base, int tid, int lognt, int M,
                                           const uint64_t *__restrict__ qdiag, float &up, float &dn,
                                           uint64_t *sH, uint64_t *sQ, uint64_t *sOut, double *s_w,
                                           Sync sync) {
  constexpr int NA = 1 << RB, NP = NA / 2;
  const uint32_t outer_par = ORIENT ? (uint32_t)(__popcll(base & d.black_outer) & 1) : 0u;
  for (int p = 0; p < d.nphases; ++p) {
    const PhaseDesc &ph = s_ph[p];
    // slot of this thread's subcube origin (host-precomputed slot of each
    // thread-index bit) and of the register bits
    uint32_t s0 = 0;
    for (int b = 0; b < lognt; ++b)
      if ((tid >> b) & 1) s0 ^= ph.tslot[b];
    uint32_t sm[RB];
#pragma unroll
    for (int k = 0; k < RB; ++k) sm[k] = ph.sm[k];
    const int o0 = ph.op0 - d.rop0;
    if (ph.nops == 1 && s_op[o0].kind == OP_DIAG) {
      diag_phase<RB, ORIENT>(tile2, d, ph, s_op[o0], base, tid, lognt, M, qdiag, sH, sQ, sOut, s0, sm, sync);
      continue;
    }
    if constexpr (ORIENT) {
      oriented_phase<RB, SITES>(tile2, d, ph, s_op + o0, base, tid, lognt, up, dn, s_w, s0, sm, outer_par);
      sync();
      continue;
    }
    // load the subcube as NP packs, walking the packs in Gray-code order so
    // each step changes one register bit (one XOR on the byte offset)
    u64 RE[NP], IM[NP];
    const char *tb = reinterpret_cast<const char *>(tile2);
    uint32_t mb[RB];
#pragma unroll
    for (int k = 0; k < RB; ++k) mb[k] = sm[k] << 3;
    const uint32_t ob = s0 << 3;
    {
      uint32_t o = ob;
#pragma unroll
      for (int g = 0; g < NP; ++g) {
        const int j = g ^ (g >> 1);
        if ((g & 7) == 0) {
          o = ob;
#pragma unroll
          for (int k = 0; k < RB - 1; ++k)
            if ((j >> k) & 1) o ^= mb[1 + k];
        } else {
          o ^= mb[1 + ctz5(g)];
        }
        const uint32_t o1 = o ^ mb[0];
        const float2 v0 = *reinterpret_cast<const float2 *>(tb + o);
        const float2 v1 = *reinterpret_cast<const float2 *>(tb + o1);
        RE[j] = pack2(v0.x, v1.x);
        IM[j] = pack2(v0.y, v1.y);
      }
    }
    ROpRes cur = s_op[o0];
    for (int k = 0; k < ph.nops; ++k) {
      const ROpRes nxt = s_op[o0 + (k + 1 < ph.nops ? k + 1 : k)];  // prefetch
      if (cur.kind == OP_GATE) {
        gate_combo(RE, IM, cur.combo, cur.t, cur.s);
      } else if (cur.kind == OP_REDUCE) {
        int kr = -1;
#pragma unroll
        for (int q = 0; q < RB; ++q)
          if (ph.rb[q] == d.site_tile) kr = q;
        uint32_t fixed_bit;
        if (d.site_tile < 0) {
          fixed_bit = (uint32_t)((base >> d.site_pos) & 1ull);
        } else {
          uint32_t t0 = 0;
          for (int b = 0; b < 5; ++b) t0 |= ((uint32_t)(tid >> b) & 1u) << ph.lanes[b];
          for (int b = 0; b < lognt - 5; ++b) t0 |= ((uint32_t)(tid >> (5 + b)) & 1u) << ph.warps[b];
          fixed_bit = (t0 >> d.site_tile) & 1u;
        }
#pragma unroll
        for (int j = 0; j < NP; ++j) {
          const float2 pr = unpack2(fma2(RE[j], RE[j], mul2(IM[j], IM[j])));
          if (kr == 0) {
            dn += pr.x;
            up += pr.y;
          } else {
            const uint32_t bit = kr > 0 ? ((uint32_t)(j >> (kr - 1)) & 1u) : fixed_bit;
            if (bit) up += pr.x + pr.y;
            else dn += pr.x + pr.y;
          }
        }
        if constexpr (SITES) {
          // per tile bit, the weight with that bit up: register bits from the
          // packs, thread-index bits the thread's whole sum
          float tsum = 0.f, ureg[RB];
#pragma unroll
          for (int q = 0; q < RB; ++q) ureg[q] = 0.f;
#pragma unroll
          for (int j = 0; j < NP; ++j) {
            const float2 pr = unpack2(fma2(RE[j], RE[j], mul2(IM[j], IM[j])));
            const float sj = pr.x + pr.y;
            tsum += sj;
            ureg[0] += pr.y;
#pragma unroll
            for (int i = 0; i < RB - 1; ++i)
              if ((j >> i) & 1) ureg[1 + i] += sj;
          }
          uint32_t tbits = 0;
          for (int b = 0; b < 5; ++b) tbits |= ((uint32_t)(tid >> b) & 1u) << ph.lanes[b];
          for (int b = 0; b < lognt - 5; ++b) tbits |= ((uint32_t)(tid >> (5 + b)) & 1u) << ph.warps[b];
#pragma unroll
          for (int q = 0; q < kMaxK; ++q) {
            float v = ((tbits >> q) & 1u) ? tsum : 0.f;
#pragma unroll
            for (int k2 = 0; k2 < RB; ++k2)
              if (ph.rb[k2] == q) v = ureg[k2];
            warp_site_sum<float>(v, q, s_w);
          }
          warp_site_sum<float>(tsum, kMaxK, s_w);
        }
      }
      cur = nxt;
    }
    {
      char *tw = reinterpret_cast<char *>(tile2);
      uint32_t o = ob;
#pragma unroll
      for (int g = 0; g < NP; ++g) {
        const int j = g ^ (g >> 1);
        if ((g & 7) == 0) {
          o = ob;
#pragma unroll
          for (int k = 0; k < RB - 1; ++k)
            if ((j >> k) & 1) o ^= mb[1 + k];
        } else {
          o ^= mb[1 + ctz5(g)];
        }
        const uint32_t o1 = o ^ mb[0];
        const float2 r = unpack2(RE[j]), i = unpack2(IM[j]);
        *reinterpret_cast<float2 *>(tw + o) = make_float2(r.x, i.x);
        *reinterpret_cast<float2 *>(tw + o1) = make_float2(r.y, i.y);
      }
    }
    sync();
  }
}

// Shared -> global store of a tile, output tile bits relabelled by perm.
// Output chunk ch = tid + nt * e of two amplitudes covers output tile index
// 2 ch: bits 1..lognt from tid, the RB - 1 high ones from e (Gray order
// again).  The amplitude there is input tile index sum of bits perm[q], so its
// slot is an XOR of per-bit slots; the chunk's second amplitude is output bit
// 0 = input bit perm[0].
template <int RB>
__device__ __forceinline__ void store_tile(float2 *psi, uint64_t base, const PassDesc &d, int tid, int lognt,
                                           const float2 *tile2) {
  constexpr int NP = 1 << (RB - 1);
  uint64_t off_lo = 0;
  uint32_t pin_lo = 0;
  for (int k = 0; k < lognt; ++k)
    if ((tid >> k) & 1) {
      const int q = d.store_bit[k];
      off_lo |= 1ull << d.tile_pos[q], pin_lo |= 1u << d.perm[q];
    }
  int64_t dh[RB - 1];
  uint32_t dsl[RB - 1];
#pragma unroll
  for (int k = 0; k < RB - 1; ++k) {
    const int q = d.store_bit[lognt + k];
    dh[k] = (int64_t)8 << d.tile_pos[q];
    dsl[k] = slot(1u << d.perm[q]) << 3;
  }
  const char *tb = reinterpret_cast<const char *>(tile2);
  const uint32_t sl1 = slot(1u << d.perm[0]) << 3;
  const uint32_t so0 = slot(pin_lo) << 3;
  char *const dst0 = reinterpret_cast<char *>(psi + base + off_lo);
  uint32_t so = so0;
  char *dst = dst0;
#pragma unroll
  for (int g = 0; g < NP; ++g) {
    if ((g & 7) == 0) {
      so = so0, dst = dst0;
#pragma unroll
      for (int k = 0; k < RB - 1; ++k)
        if (((g ^ (g >> 1)) >> k) & 1) dst += dh[k], so ^= dsl[k];
    } else {
      const int k = ctz5(g);
      dst += gray_up(g) ? dh[k] : -dh[k];
      so ^= dsl[k];
    }
    const float2 v0 = *reinterpret_cast<const float2 *>(tb + so);
    const float2 v1 = *reinterpret_cast<const float2 *>(tb + (so ^ sl1));
    *reinterpret_cast<float4 *>(dst) = make_float4(v0.x, v0.y, v1.x, v1.y);
  }
}

}  // namespace sw2

// Register-blocked sweep with RB register bits (2^RB amplitudes per thread,
// 2^(K-RB) threads per tile), one tile per block.  ORIENT: an oriented
// program on an oriented state (see Orientation).
template <int RB, bool SITES, bool ORIENT>
__global__ void __launch_bounds__(RB == 5 ? 512 : 256)
sweep2_kernel(const JobPtrs *__restrict__ jobs, float2 *psi1, const ROpRes *sops1,
              const __grid_constant__ PassDesc d, const PhaseDesc *__restrict__ phases, int M,
              unsigned ahead) {
  // one job (gridDim.y == 1): its amplitude and op arrays come with the launch
  // so the tile copies can start at once; the rest of the job's pointers
  // (and everything for a batch) from the job table
  const bool one = gridDim.y == 1;
  const JobPtrs jp = jobs[blockIdx.y];
  float2 *__restrict__ psi = one ? psi1 : static_cast<float2 *>(jp.psi);
  extern __shared__ __align__(16) float2 tile2[];
  __shared__ uint64_t sH[kMaxK];
  __shared__ uint64_t sQ[kMaxK * kMaxK];
  __shared__ uint64_t sOut;
  __shared__ __align__(16) PhaseDesc s_ph[kMaxPassPhases];
  __shared__ __align__(16) ROpRes s_op[kMaxPassOps];
  __shared__ double s_w[SITES ? kMaxWarps * kSiteSlots : 1];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lognt = d.K - RB;
  const uint64_t base = sw2::tile_origin(blockIdx.x, d, M);
  // the tile's copies first, then the pass's program (coefficients already
  // resolved for this dt), then the L2 prefetch of the tile of block
  // blockIdx.x + ahead (ahead = blocks resident at once): DRAM keeps
  // streaming while tiles compute, and that block's copies find its tile in L2
  sw2::load_tile<RB>(psi, base, d, tid, lognt, (uint32_t)__cvta_generic_to_shared(tile2));
  {
    const uint32_t *pw = reinterpret_cast<const uint32_t *>(phases + d.phase0);
    const uint32_t a_ph = (uint32_t)__cvta_generic_to_shared(s_ph);
    const int nw = d.nphases * (int)(sizeof(PhaseDesc) / 4);
    for (int i = tid; i < nw; i += nt) sw2::cp_async4(a_ph + 4u * i, pw + i);
    const ROpRes *so = (one ? sops1 : jp.sops) + d.rop0;
    const uint32_t a_op = (uint32_t)__cvta_generic_to_shared(s_op);
    for (int i = tid; i < d.nrops; i += nt) sw2::cp_async16(a_op + 16u * i, so + i);
  }
  if (ahead && blockIdx.x + ahead < gridDim.x)
    sw2::prefetch_tile<RB>(psi, sw2::tile_origin(blockIdx.x + ahead, d, M), d, tid, lognt);
  sw2::cp_async_wait_all();
  __syncthreads();

  float up = 0.f, dn = 0.f;
  sw2::run_phases<RB, SITES, ORIENT>(tile2, d, s_ph, s_op, base, tid, lognt, M, jp.qdiag, up, dn, sH, sQ,
                                     &sOut, s_w, sw2::SyncBlock{});
  sw2::store_tile<RB>(psi, base, d, tid, lognt, tile2);
  if constexpr (SITES)
    if (d.has_reduce) write_site_partials(d, M, base, s_w, jp.psites);
  if (d.has_reduce) reduce_finalize((double)up, (double)dn, jp, false);
}

// ===========================================================================
// Whole states resident in shared memory.  When one tile holds the whole
// state (K = M, one segment), every Trotter step is one pass over that tile,
// so a block can keep the state in shared memory for all the steps of an
// evolve call: one global load at the start, one store at the end, and the
// P / norm readout after every step reduced inside the block.
// ===========================================================================
// The four passes of a one-tile plan: the first, steady and last step of an
// evolve call of two or more steps, and the step of a one-step call.
struct ResidentPasses {
  PassDesc first, mid, last, only;
};

// One block per job (blockIdx.y); 2^(M-RB) threads.  Dynamic shared memory:
// the state (8 B x 2^M), then the plan's phase program (nph PhaseDesc) and its
// resolved ops (nrops ROpRes).  ORIENT: oriented program and state.
template <int RB, bool ORIENT>
__global__ void __launch_bounds__(256)
resident_kernel(const JobPtrs *__restrict__ jobs, const __grid_constant__ ResidentPasses rp,
                const PhaseDesc *__restrict__ phases, int nph, int nrops, int M, int64_t steps) {
  const JobPtrs jp = jobs[blockIdx.y];
  float2 *__restrict__ psi = static_cast<float2 *>(jp.psi);
  extern __shared__ __align__(16) float2 tile2[];
  PhaseDesc *s_ph = reinterpret_cast<PhaseDesc *>(tile2 + (size_t(1) << M));
  ROpRes *s_op = reinterpret_cast<ROpRes *>(s_ph + nph);
  __shared__ uint64_t sH[kMaxK];
  __shared__ uint64_t sQ[kMaxK * kMaxK];
  __shared__ uint64_t sOut;
  __shared__ double s_up[8], s_dn[8];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lognt = M - RB;
  // the state (tile bits = physical bits: base 0, no relabelling), then the program
  sw2::load_tile<RB>(psi, 0, rp.first, tid, lognt, (uint32_t)__cvta_generic_to_shared(tile2));
  {
    const uint32_t *pw = reinterpret_cast<const uint32_t *>(phases);
    const uint32_t a_ph = (uint32_t)__cvta_generic_to_shared(s_ph);
    const int nw = nph * (int)(sizeof(PhaseDesc) / 4);
    for (int i = tid; i < nw; i += nt) sw2::cp_async4(a_ph + 4u * i, pw + i);
    const uint32_t a_op = (uint32_t)__cvta_generic_to_shared(s_op);
    for (int i = tid; i < nrops; i += nt) sw2::cp_async16(a_op + 16u * i, jp.sops + i);
  }
  sw2::cp_async_wait_all();
  __syncthreads();
  const int64_t slot0 = *jp.step;
  const int warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
  for (int64_t k = 0; k < steps; ++k) {
    const PassDesc &d = steps == 1 ? rp.only : k == 0 ? rp.first : k == steps - 1 ? rp.last : rp.mid;
    float up = 0.f, dn = 0.f;
    sw2::run_phases<RB, false, ORIENT>(tile2, d, s_ph + d.phase0, s_op + d.rop0, 0ull, tid, lognt, M,
                                       jp.qdiag, up, dn, sH, sQ, &sOut, nullptr, sw2::SyncBlock{});
    // this step's N_up / N_dn: FP64 sums over the block in a fixed order
    double u = up, w = dn;
    for (int o = 16; o; o >>= 1) {
      u += __shfl_xor_sync(0xffffffffu, u, o);
      w += __shfl_xor_sync(0xffffffffu, w, o);
    }
    if (lane == 0) s_up[warp] = u, s_dn[warp] = w;
    __syncthreads();
    if (tid == 0) {
      double U = 0.0, D = 0.0;
      for (int i = 0; i < nw; ++i) U += s_up[i], D += s_dn[i];
      jp.series[2 * (slot0 + k)] = (U - D) / (U + D);
      jp.series[2 * (slot0 + k) + 1] = U + D;
    }
    __syncthreads();
  }
  sw2::store_tile<RB>(psi, 0, rp.first, tid, lognt, tile2);
  if (tid == 0) *jp.step = slot0 + steps;
}

}  // namespace spinrp
