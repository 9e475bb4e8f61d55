// sweep2d.cuh -- register-blocked tile sweep for complex128 states (sm_103a).
//
// The complex128 counterpart of sweep2_kernel: the same pass programs (phases
// of register bits, gates as three shears per plane, the diagonal phase by
// Gray-code field updates, the fused P/norm readout), with 32 FP64 amplitudes
// per thread and 16-byte shared-memory slots.  Bound by the FP64 pipe.
#pragma once
#include "kernels.cuh"

namespace spinrp {

// ===========================================================================
// Register-blocked sweep (complex128).  Each thread holds the 32 amplitudes of
// a five-bit subcube as FP64 real and imaginary parts.  The tile lives in
// shared memory as 16-byte amplitudes with a three-bit XOR swizzle (sw2d::slot),
// so one 16-byte access moves one amplitude and the eight lanes of an access
// quarter (three lane bits of distinct residues mod 3) hit distinct 16-byte
// bank groups.  Gates are the same three shears per plane as shear_rotate.
// ===========================================================================
namespace sw2d {

// Shared-memory slot (16-byte units) of tile index t: the low three bits
// XORed with bits 3-5, 6-8, 9-11 and 12-14.  XOR-linear.
__device__ __forceinline__ uint32_t slot(uint32_t t) {
  return t ^ (((t >> 3) ^ (t >> 6) ^ (t >> 9) ^ (t >> 12)) & 7u);
}

// Gate on register bits (KU, KV) of the thread's 32 amplitudes: planes
// (re a, im b) and (re b, im a) for a = bit KU set / KV clear, b = the reverse.
template <int KU, int KV>
__device__ __forceinline__ void gate(double (&re)[32], double (&im)[32], double t, double s) {
#pragma unroll
  for (int i = 0; i < 32; ++i)
    if (((i >> KU) & 1) == 1 && ((i >> KV) & 1) == 0) {
      const int k = i ^ (1 << KU) ^ (1 << KV);
      double x = fma(t, im[k], re[i]);
      im[k] = fma(-s, x, im[k]);
      re[i] = fma(t, im[k], x);
      x = fma(t, im[i], re[k]);
      im[i] = fma(-s, x, im[i]);
      re[k] = fma(t, im[i], x);
    }
}

// combo = index of (ku < kv) among the ten register-bit pairs, lexicographic.
__device__ __forceinline__ void gate_combo(double (&re)[32], double (&im)[32], int combo, double t, double s) {
  switch (combo) {
    case 0: gate<0, 1>(re, im, t, s); break;
    case 1: gate<0, 2>(re, im, t, s); break;
    case 2: gate<0, 3>(re, im, t, s); break;
    case 3: gate<0, 4>(re, im, t, s); break;
    case 4: gate<1, 2>(re, im, t, s); break;
    case 5: gate<1, 3>(re, im, t, s); break;
    case 6: gate<1, 4>(re, im, t, s); break;
    case 7: gate<2, 3>(re, im, t, s); break;
    case 8: gate<2, 4>(re, im, t, s); break;
    default: gate<3, 4>(re, im, t, s); break;
  }
}

// A phase op staged in shared memory with its FP64 gate coefficients.
struct SOpD {
  uint8_t kind, combo, arg, pad[5];
  double t, s;
};

}  // namespace sw2d

// at most 2^13-amplitude tiles: 256 threads
__global__ void __launch_bounds__(256)
sweep2d_kernel(const JobPtrs *__restrict__ jobs, const __grid_constant__ PassDesc d,
               const PhaseDesc *__restrict__ phases, const ROp *__restrict__ rops, int M, unsigned ahead) {
  constexpr int RB = 5, NA = 32;
  const JobPtrs jp = jobs[blockIdx.y];
  double2 *__restrict__ psi = static_cast<double2 *>(jp.psi);
  const uint64_t *__restrict__ qdiag = jp.qdiag;
  extern __shared__ __align__(16) double2 tile16[];
  __shared__ uint64_t sH[kMaxK];
  __shared__ uint64_t sQ[kMaxK * kMaxK];
  __shared__ uint64_t sOut;
  __shared__ PhaseDesc s_ph[kMaxPassPhases];
  __shared__ sw2d::SOpD s_op[kMaxPassOps];
  const int K = d.K, tid = threadIdx.x, nt = blockDim.x;
  const int lognt = K - RB;
  const uint64_t base = sw2::tile_origin(blockIdx.x, d, M);
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(tile16);
  // ---- global -> shared: 16-byte async copies, amplitude a = tid + nt * e,
  // e in Gray-code order in runs of eight (as in the complex64 kernel)
  {
    uint64_t off_lo = 0;
    for (int k = 0; k < lognt; ++k)
      if ((tid >> k) & 1) off_lo |= 1ull << d.tile_pos[k];
    int64_t dg[RB];
    uint32_t ds[RB];
#pragma unroll
    for (int k = 0; k < RB; ++k) {
      dg[k] = (int64_t)16 << d.tile_pos[lognt + k];
      ds[k] = sw2d::slot(1u << (lognt + k)) << 4;
    }
    const char *src0 = reinterpret_cast<const char *>(psi + base + off_lo);
    const uint32_t sb0 = sw2d::slot((uint32_t)tid) << 4;
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
        const int k = sw2::ctz5(g);
        src += sw2::gray_up(g) ? dg[k] : -dg[k];
        sb ^= ds[k];
      }
      sw2::cp_async16(sbase + sb, src);
    }
  }
  // the pass's program; FP64 coefficients from the job's table
  for (int i = tid; i < d.nphases; i += nt) s_ph[i] = phases[d.phase0 + i];
  for (int i = tid; i < d.nrops; i += nt) {
    const ROp r = rops[d.rop0 + i];
    sw2d::SOpD o;
    o.kind = r.kind, o.combo = r.combo, o.arg = r.arg;
    o.t = 0.0, o.s = 0.0;
    if (r.kind == OP_GATE) {
      const GateCoef g = jp.coefs[r.coef];
      o.t = g.t, o.s = g.s;
    }
    s_op[i] = o;
  }
  // L2 prefetch of the tile of block blockIdx.x + ahead (128-byte runs: tile
  // bits 0..2, the low physical bits)
  if (ahead && blockIdx.x + ahead < gridDim.x) {
    uint64_t ot = sw2::tile_origin(blockIdx.x + ahead, d, M);
    for (int b = 0; b < lognt; ++b)
      if ((tid >> b) & 1) ot |= 1ull << d.tile_pos[3 + b];
#pragma unroll
    for (int i = 0; i < (1 << (RB - 3)); ++i) {
      uint64_t off = ot;
#pragma unroll
      for (int b = 0; b < RB - 3; ++b)
        if ((i >> b) & 1) off |= 1ull << d.tile_pos[3 + lognt + b];
      asm volatile("prefetch.global.L2 [%0];" ::"l"(psi + off));
    }
  }
  sw2::cp_async_wait_all();
  __syncthreads();

  double up = 0.0, dn = 0.0;
  const int nout = M - K;
  const char *tb = reinterpret_cast<const char *>(tile16);
  char *tw = reinterpret_cast<char *>(tile16);
  for (int p = 0; p < d.nphases; ++p) {
    const PhaseDesc &ph = s_ph[p];
    uint32_t s0 = 0;  // slot of the subcube origin
    for (int b = 0; b < lognt; ++b)
      if ((tid >> b) & 1) s0 ^= ph.tslot[b];
    uint32_t sm[RB];
#pragma unroll
    for (int k = 0; k < RB; ++k) sm[k] = ph.sm[k];
    const int o0 = ph.op0 - d.rop0;
    uint32_t t0 = 0;  // tile bits from the thread index
    for (int k = 0; k < 5; ++k) t0 |= ((uint32_t)(tid >> k) & 1u) << ph.lanes[k];
    for (int k = 0; k < lognt - 5; ++k) t0 |= ((uint32_t)(tid >> (5 + k)) & 1u) << ph.warps[k];
    if (ph.nops == 1 && s_op[o0].kind == OP_DIAG) {
      // e^{-i tau D} amplitude by amplitude in shared memory, Theta walked in
      // Gray-code order over the register bits (as in the complex64 kernel)
      const uint64_t *q = qdiag + (size_t)s_op[o0].arg * M * M;
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
        uint64_t sacc = 0;
        for (int o = 0; o < nout; ++o)
          for (int o2 = o + 1; o2 < nout; ++o2) {
            const int pa = d.outer_pos[o], pb = d.outer_pos[o2];
            const uint64_t v = q[pa * M + pb];
            sacc += (((base >> pa) ^ (base >> pb)) & 1ull) ? (0ull - v) : v;
          }
        sOut = sacc;
      }
      for (int w = tid; w < K * K; w += nt) sQ[w] = q[d.tile_pos[w / K] * M + d.tile_pos[w % K]];
      __syncthreads();
      uint32_t isreg = 0;
      for (int k = 0; k < RB; ++k) isreg |= 1u << ph.rb[k];
      uint64_t th0 = sOut;
      for (int x = 0; x < K; ++x) {
        if ((isreg >> x) & 1u) continue;
        const uint32_t bx = (t0 >> x) & 1u;
        th0 += bx ? sH[x] : (0ull - sH[x]);
        for (int y = x + 1; y < K; ++y) {
          if ((isreg >> y) & 1u) continue;
          th0 += (bx ^ ((t0 >> y) & 1u)) ? (0ull - sQ[x * K + y]) : sQ[x * K + y];
        }
      }
      uint64_t G[RB], Qr[RB][RB], F[RB];
#pragma unroll
      for (int k = 0; k < RB; ++k) {
        const int rk = ph.rb[k];
        uint64_t gk = sH[rk];
        for (int x = 0; x < K; ++x) {
          if ((isreg >> x) & 1u) continue;
          gk += ((t0 >> x) & 1u) ? sQ[x * K + rk] : (0ull - sQ[x * K + rk]);
        }
        G[k] = gk;
      }
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
      uint32_t sl = s0;
#pragma unroll
      for (int g = 0; g < NA; ++g) {
        if (g) {
          const int k = sw2::ctz5(g);
          const bool was_up = ((((g - 1) ^ ((g - 1) >> 1)) >> k) & 1) != 0;
          th += was_up ? (0ull - 2ull * F[k]) : 2ull * F[k];
#pragma unroll
          for (int l = 0; l < RB; ++l)
            if (l != k) F[l] += was_up ? (0ull - 2ull * Qr[l][k]) : 2ull * Qr[l][k];
          sl ^= sm[k];
        }
        tile16[sl] = cmul(tile16[sl], cis_turns(th, 0.0));
      }
      __syncthreads();
      continue;
    }
    // the subcube, one 16-byte amplitude per access, Gray-code walk over the
    // five register bits in runs of eight
    double re[NA], im[NA];
    const uint32_t ob = s0 << 4;
    {
      uint32_t o = ob;
#pragma unroll
      for (int g = 0; g < NA; ++g) {
        const int j = g ^ (g >> 1);
        if ((g & 7) == 0) {
          o = ob;
#pragma unroll
          for (int k = 0; k < RB; ++k)
            if ((j >> k) & 1) o ^= sm[k] << 4;
        } else {
          o ^= sm[sw2::ctz5(g)] << 4;
        }
        const double2 v = *reinterpret_cast<const double2 *>(tb + o);
        re[j] = v.x;
        im[j] = v.y;
      }
    }
    for (int k = 0; k < ph.nops; ++k) {
      const sw2d::SOpD &op = s_op[o0 + k];
      if (op.kind == OP_GATE) {
        sw2d::gate_combo(re, im, op.combo, op.t, op.s);
      } else if (op.kind == OP_REDUCE) {
        int kr = -1;
#pragma unroll
        for (int qq = 0; qq < RB; ++qq)
          if (ph.rb[qq] == d.site_tile) kr = qq;
        const uint32_t fixed_bit = d.site_tile < 0 ? (uint32_t)((base >> d.site_pos) & 1ull)
                                                   : ((t0 >> d.site_tile) & 1u);
#pragma unroll
        for (int j = 0; j < NA; ++j) {
          const double pr = re[j] * re[j] + im[j] * im[j];
          const uint32_t bit = kr >= 0 ? ((uint32_t)(j >> kr) & 1u) : fixed_bit;
          if (bit) up += pr;
          else dn += pr;
        }
      }
    }
    {
      uint32_t o = ob;
#pragma unroll
      for (int g = 0; g < NA; ++g) {
        const int j = g ^ (g >> 1);
        if ((g & 7) == 0) {
          o = ob;
#pragma unroll
          for (int k = 0; k < RB; ++k)
            if ((j >> k) & 1) o ^= sm[k] << 4;
        } else {
          o ^= sm[sw2::ctz5(g)] << 4;
        }
        *reinterpret_cast<double2 *>(tw + o) = make_double2(re[j], im[j]);
      }
    }
    __syncthreads();
  }

  // ---- shared -> global: output amplitude tid + nt * e (tile bits 0..lognt-1
  // from tid) takes the amplitude of input tile index sum of bits perm[q]
  {
    uint64_t off_lo = 0;
    uint32_t pin_lo = 0;
    for (int k = 0; k < lognt; ++k)
      if ((tid >> k) & 1) off_lo |= 1ull << d.tile_pos[k], pin_lo |= 1u << d.perm[k];
    int64_t dh[RB];
    uint32_t dsl[RB];
#pragma unroll
    for (int k = 0; k < RB; ++k) {
      dh[k] = (int64_t)16 << d.tile_pos[lognt + k];
      dsl[k] = sw2d::slot(1u << d.perm[lognt + k]) << 4;
    }
    const uint32_t so0 = sw2d::slot(pin_lo) << 4;
    char *const dst0 = reinterpret_cast<char *>(psi + base + off_lo);
    uint32_t so = so0;
    char *dst = dst0;
#pragma unroll
    for (int g = 0; g < NA; ++g) {
      if ((g & 7) == 0) {
        so = so0, dst = dst0;
#pragma unroll
        for (int k = 0; k < RB; ++k)
          if (((g ^ (g >> 1)) >> k) & 1) dst += dh[k], so ^= dsl[k];
      } else {
        const int k = sw2::ctz5(g);
        dst += sw2::gray_up(g) ? dh[k] : -dh[k];
        so ^= dsl[k];
      }
      *reinterpret_cast<double2 *>(dst) = *reinterpret_cast<const double2 *>(tb + so);
    }
  }
  if (d.has_reduce) reduce_finalize(up, dn, jp, false);
}

}  // namespace spinrp
