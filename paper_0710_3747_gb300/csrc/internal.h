// internal.h -- structures shared by the host planner and the device kernels.
#pragma once
#include <stdint.h>
#include <vector_types.h>

#include <string>
#include <utility>
#include <vector>

namespace spinrp {

constexpr int kMaxM = 34;   // largest system (2^34 c64 amplitudes = 128 GiB)
constexpr int kMaxK = 14;   // widest shared-memory tile (2^14 c64 = 128 KiB)

enum OpKind : uint8_t {
  OP_GATE = 1,    // flip-flop gate on tile-local bits (u, v), coefficient index `coef`
  OP_DIAG = 2,    // e^{-i tau D} on every amplitude of the tile, tau variant `arg`
  OP_REDUCE = 3,  // accumulate N_up / N_dn of the readout spin into this pass's slot
};

// One operation of a sweep, in tile-local bit indices.
struct Op {
  uint8_t kind;
  uint8_t u, v;   // tile-local bits of a gate
  uint8_t arg;    // diagonal variant (0: dt/2, 1: dt)
  int32_t coef;   // gate coefficient index = 2*bond + variant (0: dt/2, 1: dt)
};

// Descriptor of one sweep ("pass") over the whole state: the state is cut into
// 2^(M-K) tiles of 2^K amplitudes; tile-local bit q sits at physical bit
// position tile_pos[q] (ascending, so tile bits 0..c-1 are the contiguous low
// bits), the block index supplies the remaining bits at outer_pos[].
struct PassDesc {
  int32_t K;
  int32_t nops;
  int32_t op0;          // first op in the global op array
  int32_t site_tile;    // tile-local bit of the readout spin, or -1 when it is an outer bit
  int32_t site_pos;     // physical position of the readout spin
  int32_t has_reduce;
  int32_t relabel;      // nonzero when the tile is written back with permuted bits
  uint8_t tile_pos[kMaxK];
  uint8_t outer_pos[kMaxM];
  uint8_t perm[kMaxK];  // store: output tile bit q takes the amplitude bit of input tile bit perm[q]
  uint8_t tile_spin[kMaxK];   // logical spin (0-based) at each tile bit, input layout
  uint8_t outer_spin[kMaxM];  // logical spin at each outer bit, input layout
  int32_t phase0;       // register-blocked program: first phase
  int32_t nphases;      //   and number of phases,
  int32_t rop0;         //   first op
  int32_t nrops;        //   and number of ops
  uint8_t store_bit[kMaxK];  // store: output tile bit (1..K-1) of each chunk-index bit
  // oriented states (see Orientation below): tile bits and outer physical
  // positions that hold spins of the first colour, input layout
  uint32_t black_tile;
  uint64_t black_outer;
};

// Register-blocked execution of a pass.  In a phase every thread holds the
// 2^RB amplitudes of the tile that differ only in the RB tile bits rb[] (its
// "subcube"; RB = 5 or 6 per plan for complex64, 5 for complex128), applies
// the phase's ops to them in registers and writes them back to shared memory.
// lanes[]/warps[] give the tile bits the thread index supplies.
constexpr int kMaxRegBits = 6;  // 5 or 6 register bits per phase
struct PhaseDesc {
  uint8_t rb[kMaxRegBits];
  uint8_t lanes[5];
  uint8_t warps[kMaxK - 10];
  uint8_t nops;
  uint8_t nb;  // oriented program: register bits 0..nb-1 hold first-colour spins
  int32_t op0;
  uint16_t sm[kMaxRegBits];  // shared-memory slot of each register bit
  uint16_t tslot[kMaxK - 5]; // slot of each thread-index bit (lanes, then warps)
  uint16_t pad2;
};

// A pass's register-blocked program is staged in shared memory; passes with
// more phases or ops than this run the plain sweep kernel instead.
constexpr int kMaxPassPhases = 96;
constexpr int kMaxPassOps = 768;

// Orientation (complex64 states of a bipartite flip-flop graph).  The spins
// are 2-coloured so that every bond joins the two colours; an amplitude whose
// basis index has an odd number of first-colour ("black") spins up is stored
// with its real and imaginary parts swapped, (Im, Re).  The two amplitudes a
// gate mixes differ in one black spin, so one is stored (Re, Im) and the
// other (Im, Re), and the gate's three shears become packed FP32x2 updates
// of the two stored words as they are (no re/im shuffling).  Each phase of an
// oriented program holds its nb black register bits first, then the others;
// nb is one of the counts kOrientNbMask(RB) allows (the kernel has gate code
// for those).
inline uint32_t kOrientNbMask(int RB) { return RB == 6 ? 0x1Cu : 0x0Cu; }  // {2,3,4} / {2,3}

// Shared-memory slot of tile index t in the register-blocked kernel: the low
// four bits are XORed with bits 4-7, 8-11 and 12-15 (XOR-linear).
inline uint32_t swizzle_slot(uint32_t t) { return t ^ (((t >> 4) ^ (t >> 8) ^ (t >> 12)) & 15u); }
// The complex128 kernel's slot, in 16-byte units: the low three bits are
// XORed with bits 3-5, 6-8, 9-11 and 12-14 (XOR-linear).
inline uint32_t swizzle_slot16(uint32_t t) { return t ^ (((t >> 3) ^ (t >> 6) ^ (t >> 9) ^ (t >> 12)) & 7u); }

// Op of a phase: GATE acts on register bits given by `combo` (index of the
// pair (ku < kv) among the RB(RB-1)/2 pairs, lexicographic; in an oriented
// program ku < nb <= kv and combo = 8 ku + kv); DIAG / REDUCE as in Op.
struct ROp {
  uint8_t kind;
  uint8_t combo;
  uint8_t arg;
  uint8_t pad;
  int32_t coef;
};

struct GateCoef;

// A phase op with its FP32 gate coefficients resolved for the current dt (one
// array per job, rebuilt with the gate table), 16 bytes for 16-byte copies.
struct ROpRes {
  uint8_t kind, combo, arg, pad;
  float t, s;  // shear coefficients tan(theta/2), sin(theta) of a gate
  uint32_t pad2;
};
static_assert(sizeof(ROpRes) == 16, "ROpRes is copied in 16-byte pieces");
static_assert(sizeof(PhaseDesc) % 4 == 0, "PhaseDesc is copied in 4-byte pieces");

// Device pointers of one job (one state) as the kernels see them; a launch
// covers gridDim.y jobs that share one sweep plan, block row y using jobs[y].
struct JobPtrs {
  void *psi;               // 2^M amplitudes (float2 or double2)
  const GateCoef *coefs;   // 2 * bonds gate coefficients (dt/2, dt)
  const uint64_t *qdiag;   // 2 * M * M fixed-point pair phases (dt/2, dt), physical indexing
  double2 *partials;       // one (N_up, N_dn) pair per block of a launch
  unsigned *ticket;        // blocks finished in the current reducing launch
  int64_t *step;           // entries recorded in `series` so far
  double *series;          // (P, norm) per recorded step
  const double *bvals;     // flip-flop coupling of each bond (for the gate tables)
  const double *a;         // M * M S^zS^z couplings, logical indexing (for the phase tables)
  double *psites;          // all-site readout: (M + 1) columns of per-block sums, column 0 the
                           // norm, column 1 + q the weight with spin q up (q logical, 0-based);
                           // nullptr when only spin 1 is read out
  double *site_series;     // all-site readout: P of spin q at entry k in site_series[k * M + q]
  ROpRes *sops;            // register-blocked program ops with resolved coefficients
};

// Gate coefficients of exp(-i theta sigma_x) on a flip-flop pair, theta = b tau/2:
// (tan theta/2, sin theta) of the three-shear form of the two real plane
// rotations the gate is made of (see shear_rotate), in FP64 and as the FP32
// pair closest to a rotation.
struct GateCoef {
  double t, s;
  float tf, sft;
};

// ---------------------------------------------------------------------------
// Host plan
// ---------------------------------------------------------------------------
struct PlanGate {
  int bond;   // index into the canonical bond list
  int i, j;   // logical spins (0-based)
};

struct Plan {
  int M = 0, K = 0, c = 0;
  std::vector<int> pos;                      // logical spin -> physical bit position
  std::vector<std::vector<PlanGate>> seg;    // forward half step cut into segments
  std::vector<std::vector<int>> segQ;        // logical spins of each segment's tile
  std::vector<std::vector<int>> exitX;       // spins moved into the low bits after segment k
  int segments() const { return (int)seg.size(); }
  int sweeps_per_step() const { return seg.size() <= 1 ? 1 : 2 * (int)seg.size() - 2; }
};

// Set the calling thread's spinrp_last_error() message; returns code.
int report_error(int code, const char *msg);

// Build the plan for the canonical bonds with tiles of K spins whose lowest c
// physical bits are shared by every tile.  Returns false and sets *err on failure.
bool build_plan(int M, const std::vector<std::pair<int, int>> &bonds, int K, int c, Plan *plan,
                std::string *err);

// Phases of a pass for the register-blocked kernel: gates (pairs of tile bits,
// in order) cut into register sets of RB of the K tile bits; sets[k] (bit
// mask) applies the gates applied[k], in an order that keeps every bit's gate
// sequence, and no gate from index `fence` on before every gate ahead of it
// (an element-wise op sits between them).  Beam search of width `beam` for
// few phases.  With nb_allowed != 0 every set holds nb bits of the mask
// `black` and RB - nb others for an nb whose bit is set in nb_allowed (the
// oriented kernel's colour patterns).  False if a gate cannot be placed.
bool plan_phases(int K, const std::vector<std::pair<int, int>> &gates, int RB, int beam, int fence,
                 std::vector<uint32_t> *sets, std::vector<std::vector<int>> *applied,
                 uint32_t black = 0, uint32_t nb_allowed = 0);

}  // namespace spinrp
