// api.cu -- C ABI (include/spinrp.h): spin systems, the sweep plan, device
// states and the evolve loop.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/spinrp.h"
#include "internal.h"
#include "kernels.cuh"
#include "persist.cuh"
#include "pipe.cuh"
#include "sectors.cuh"
#include "sweep2d.cuh"

using namespace spinrp;

// ---------------------------------------------------------------------------
// error reporting
// ---------------------------------------------------------------------------
static thread_local std::string g_err;

static int fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

// Error reporting for the other translation units of the library.
int spinrp::report_error(int code, const char *msg) {
  g_err = msg;
  return code;
}

#define CUDA_TRY(call)                                                                 \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) return fail(SPINRP_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

static std::atomic<int64_t> g_launches{0};

extern "C" const char *spinrp_last_error(void) { return g_err.c_str(); }
extern "C" int64_t spinrp_launch_count(void) { return g_launches.load(); }
extern "C" const char *spinrp_version(void) { return "spinrp 0.1 (sm_103a)"; }

// ---------------------------------------------------------------------------
// systems
// ---------------------------------------------------------------------------
struct spinrp_system {
  int M = 0, htype = 0;
  std::vector<double> a, b;  // M*M, symmetric, zero diagonal
  std::vector<std::pair<int, int>> bonds;
  int tileK[2] = {0, 0};
  int regbits = 0;  // register bits per phase of the complex64 kernel (0: default)
  // 2-colouring of the flip-flop graph (every bond joins the colours), when
  // one exists: mask of the first-colour spins (see Orientation)
  bool bipartite = false;
  uint64_t black = 0;
  int orient_mode = 0;  // 1: complex64 states are oriented when they can be; 0: never
};

// Colour the spins of the flip-flop graph with two colours so that every bond
// joins them (breadth first from each uncoloured spin); false if an odd cycle
// makes that impossible.  The first colour ("black") is the smaller class.
static bool two_colour(int M, const std::vector<std::pair<int, int>> &bonds, uint64_t *black) {
  std::vector<std::vector<int>> adj(M);
  for (auto &b : bonds) adj[b.first].push_back(b.second), adj[b.second].push_back(b.first);
  std::vector<int> col(M, -1), queue;
  for (int r = 0; r < M; ++r) {
    if (col[r] >= 0) continue;
    col[r] = 0;
    queue.assign(1, r);
    for (size_t h = 0; h < queue.size(); ++h) {
      const int x = queue[h];
      for (int y : adj[x]) {
        if (col[y] < 0) col[y] = 1 - col[x], queue.push_back(y);
        else if (col[y] == col[x]) return false;
      }
    }
  }
  int n1 = 0;
  for (int q = 0; q < M; ++q) n1 += col[q];
  const int want = 2 * n1 <= M ? 1 : 0;
  uint64_t m = 0;
  for (int q = 0; q < M; ++q)
    if (col[q] == want) m |= 1ull << q;
  *black = m;
  return true;
}

static bool any_diag(const spinrp_system &s) {
  for (int i = 0; i < s.M; ++i)
    for (int j = i + 1; j < s.M; ++j)
      if (s.a[i * s.M + j] != 0.0) return true;
  return false;
}

extern "C" int spinrp_system_create(int M, const double *J, int htype, const double *a_generic,
                                    spinrp_system **out) {
  if (!out) return fail(SPINRP_EINVAL, "system_create: out is NULL");
  *out = nullptr;
  if (M < 2 || M > kMaxM) return fail(SPINRP_EINVAL, "system_create: M=%d outside 2..%d", M, kMaxM);
  if (!J) return fail(SPINRP_EINVAL, "system_create: J is NULL");
  if (htype < SPINRP_XY || htype > SPINRP_GENERIC)
    return fail(SPINRP_EINVAL, "system_create: unknown Hamiltonian type %d", htype);
  if (htype == SPINRP_GENERIC && !a_generic)
    return fail(SPINRP_EINVAL, "system_create: GENERIC needs a_generic");
  spinrp_system *s = new (std::nothrow) spinrp_system;
  if (!s) return fail(SPINRP_ENOMEM, "system_create: out of host memory");
  s->M = M;
  s->htype = htype;
  s->a.assign(M * M, 0.0);
  s->b.assign(M * M, 0.0);
  for (int i = 0; i < M; ++i)
    for (int j = i + 1; j < M; ++j) {
      const double Jij = J[i * M + j];
      const double ag = a_generic ? a_generic[i * M + j] : 0.0;
      if (!std::isfinite(Jij) || !std::isfinite(ag)) {
        delete s;
        return fail(SPINRP_EINVAL, "system_create: non-finite coupling at (%d,%d)", i + 1, j + 1);
      }
      double aij = 0.0, bij = 0.0;
      switch (htype) {
        case SPINRP_XY: bij = Jij; break;
        case SPINRP_DIPOLAR: aij = 2.0 * Jij, bij = -Jij; break;
        case SPINRP_ISOTROPIC: aij = Jij, bij = Jij; break;
        case SPINRP_ISING: aij = Jij; break;
        default: aij = ag, bij = Jij; break;
      }
      s->a[i * M + j] = s->a[j * M + i] = aij;
      s->b[i * M + j] = s->b[j * M + i] = bij;
    }
  for (int i = 0; i < M; ++i)
    for (int j = i + 1; j < M; ++j)
      if (s->b[i * M + j] != 0.0) s->bonds.push_back({i, j});
  s->bipartite = two_colour(M, s->bonds, &s->black);
  *out = s;
  return SPINRP_OK;
}

extern "C" int spinrp_ladder_create(int L, double j_leg, double j_rung, spinrp_system **out) {
  if (L < 1 || 2 * L > kMaxM || !std::isfinite(j_leg) || !std::isfinite(j_rung))
    return fail(SPINRP_EINVAL, "ladder_create: bad argument (L=%d)", L);
  const int M = 2 * L;
  std::vector<double> J((size_t)M * M, 0.0);
  for (int k = 0; k + 1 < L; ++k) {
    J[k * M + k + 1] = J[(k + 1) * M + k] = j_leg;                                  // leg 1..L
    J[(L + k) * M + L + k + 1] = J[(L + k + 1) * M + L + k] = j_leg;                // leg L+1..2L
  }
  for (int k = 0; k < L; ++k) J[k * M + L + k] = J[(L + k) * M + k] = j_rung;  // rungs (n, n+L)
  return spinrp_system_create(M, J.data(), SPINRP_XY, nullptr, out);
}

namespace {
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11), host side: the star's
// geometry draws.
void host_philox(uint32_t c[4], uint32_t k0, uint32_t k1) {
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c[0], p1 = (uint64_t)0xCD9E8D57u * c[2];
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k0, n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k1;
    c[1] = (uint32_t)p1, c[3] = (uint32_t)p0, c[0] = n0, c[2] = n2;
    k0 += 0x9E3779B9u, k1 += 0xBB67AE85u;
  }
}
// u in [0, 1) from two 32-bit words (top 53 bits)
double host_u53(uint32_t hi, uint32_t lo) {
  return (double)((((uint64_t)hi << 32) | lo) >> 11) * (1.0 / 9007199254740992.0);
}
}  // namespace

extern "C" int spinrp_star_dipolar_create(int M, uint64_t geom_seed, double rmin, spinrp_system **out) {
  if (M < 2 || M > kMaxM || !(rmin >= 0.0) || rmin > 0.5)
    return fail(SPINRP_EINVAL, "star_dipolar_create: bad argument (M=%d, rmin=%g)", M, rmin);
  // spin 1 at the origin; candidates n = 0, 1, ...: counter (n, 0, 0, 2)
  // gives x, y from words (0,1), (2,3), counter (n, 1, 0, 2) gives z; a
  // candidate outside the unit ball or closer than rmin to a kept spin is
  // dropped
  const uint32_t k0 = (uint32_t)geom_seed, k1 = (uint32_t)(geom_seed >> 32);
  std::vector<double> px(1, 0.0), py(1, 0.0), pz(1, 0.0);
  for (uint32_t n = 0; (int)px.size() < M; ++n) {
    if (n > 100000000u) return fail(SPINRP_EINVAL, "star_dipolar_create: cannot place %d spins", M);
    uint32_t a[4] = {n, 0u, 0u, 2u}, b[4] = {n, 1u, 0u, 2u};
    host_philox(a, k0, k1);
    host_philox(b, k0, k1);
    const double x = 2.0 * host_u53(a[0], a[1]) - 1.0, y = 2.0 * host_u53(a[2], a[3]) - 1.0,
                 z = 2.0 * host_u53(b[0], b[1]) - 1.0;
    if (x * x + y * y + z * z > 1.0) continue;
    bool ok = true;
    for (size_t q = 0; q < px.size() && ok; ++q) {
      const double dx = x - px[q], dy = y - py[q], dz = z - pz[q];
      ok = dx * dx + dy * dy + dz * dz >= rmin * rmin;
    }
    if (ok) px.push_back(x), py.push_back(y), pz.push_back(z);
  }
  // J_ij = (1 - 3 cos^2 theta_ij) / r_ij^3 (theta from the z axis), unit rms over pairs
  std::vector<double> J((size_t)M * M, 0.0);
  double sum2 = 0.0;
  for (int i = 0; i < M; ++i)
    for (int j = i + 1; j < M; ++j) {
      const double dx = px[i] - px[j], dy = py[i] - py[j], dz = pz[i] - pz[j];
      const double r2 = dx * dx + dy * dy + dz * dz, r = std::sqrt(r2);
      const double c = dz / r, v = (1.0 - 3.0 * c * c) / (r2 * r);
      J[i * M + j] = J[j * M + i] = v;
      sum2 += v * v;
    }
  const double rms = std::sqrt(sum2 / (0.5 * M * (M - 1)));
  for (double &v : J) v /= rms;
  return spinrp_system_create(M, J.data(), SPINRP_DIPOLAR, nullptr, out);
}

extern "C" int spinrp_system_couplings(const spinrp_system *sys, double *a, double *b) {
  if (!sys || (!a && !b)) return fail(SPINRP_EINVAL, "system_couplings: bad argument");
  if (a) std::copy(sys->a.begin(), sys->a.end(), a);
  if (b) std::copy(sys->b.begin(), sys->b.end(), b);
  return SPINRP_OK;
}

extern "C" int spinrp_schedule(const spinrp_system *sys, int32_t *bond_order, int cap, int *n) {
  if (!sys || !n || (cap > 0 && !bond_order)) return fail(SPINRP_EINVAL, "schedule: bad argument");
  *n = (int)sys->bonds.size();
  for (int k = 0; k < std::min(cap, *n); ++k) bond_order[k] = k;
  return SPINRP_OK;
}

extern "C" void spinrp_system_destroy(spinrp_system *sys) { delete sys; }

extern "C" int spinrp_system_num_spins(const spinrp_system *sys) { return sys ? sys->M : 0; }

extern "C" int spinrp_system_bonds(const spinrp_system *sys, int32_t *pairs, int cap, int *n) {
  if (!sys || !n || (cap > 0 && !pairs)) return fail(SPINRP_EINVAL, "system_bonds: bad argument");
  *n = (int)sys->bonds.size();
  for (int k = 0; k < std::min(cap, *n); ++k) {
    pairs[2 * k] = sys->bonds[k].first + 1;
    pairs[2 * k + 1] = sys->bonds[k].second + 1;
  }
  return SPINRP_OK;
}

// Default tile width for complex128: the widest K <= 12 that still gives at
// least 128 tiles (every SM's FP64 pipe busy), at least 8: 12 for states of
// 19+ spins (64 KiB tiles, two per SM, the register-blocked FP64 sweep at the
// FP64 pipe's rate), narrower below; 2^8-amplitude tiles (per-gate kernel) for
// 15 spins and fewer.  Measured on GB300 (us per step, this rule's pick first):
// 2x6 ladder K8 28.1 against K12 71.5; 14-spin star K8 140.6 against K12
// 397.2; 2x8 ladder K9 47.5 against K12 98.2 (K8 44.3); 2x9 ladder K11 ~ K12;
// 20- and 22-spin stars and the 2x15 ladder K12 fastest.  complex64 picks
// among 12, 13 and 14 spins by the cost model in make_plan.
static int c128_tile(int M) {
  for (int K = 12; K >= 8; --K)
    if (M - K >= 7) return K;
  return std::min(8, M);
}
static int low_bits(int prec) { return prec == SPINRP_C64 ? 4 : 3; }  // 128-byte runs

extern "C" int spinrp_system_set_tile(spinrp_system *sys, int prec, int K) {
  if (!sys || (prec != SPINRP_C64 && prec != SPINRP_C128))
    return fail(SPINRP_EINVAL, "system_set_tile: bad argument");
  const int kmax = prec == SPINRP_C64 ? 14 : 13;
  if (K < 0 || K > kmax) return fail(SPINRP_EINVAL, "system_set_tile: K=%d outside 0..%d", K, kmax);
  sys->tileK[prec] = K;
  return SPINRP_OK;
}

extern "C" int spinrp_system_set_orientation(spinrp_system *sys, int mode) {
  if (!sys || (mode != 0 && mode != 1))
    return fail(SPINRP_EINVAL, "system_set_orientation: mode must be 0 or 1");
  sys->orient_mode = mode;
  return SPINRP_OK;
}

extern "C" int spinrp_system_set_regbits(spinrp_system *sys, int rb) {
  if (!sys || !(rb == 0 || rb == 5 || rb == 6))
    return fail(SPINRP_EINVAL, "system_set_regbits: rb must be 0, 5 or 6");
  sys->regbits = rb;
  return SPINRP_OK;
}

// The plan for precision prec.  An explicit tile width (set_tile) is used as
// given; otherwise complex64 states take the tile width K in {14, 13, 12}
// (at most M) of least modelled cost, sweeps per step x max(2^K, njobs 2^M /
// kModelSMs): a sweep lasts about one tile's work while the tiles do not fill
// the SMs, and about the state's share per SM once they do.  Ties go to 13,
// then 12, then 14.  Measured on GB300 against the other widths: ladders of
// 14, 18, 22, 24 and 30 spins, dipolar stars of 16, 20 and 22 spins, and the
// batch of 12..22-spin stars (the model's pick was the fastest, or within
// 2 %, in every case).  Where 13-spin tiles run as the pipelined sweep
// (pipe_kernel: six register bits, plain storage, at least four units per
// SM) a sweep costs kPipeSweepCost of the model's sweep: measured per-sweep
// time of the pipelined 13-spin sweep over the 14-spin one 0.58, 0.59 and
// 0.72 on dipolar stars of 23, 24 and 26 spins, 0.48, 0.70 and 0.67 on
// ladders of 24, 26 and 28 spins, 0.49 and 0.47 on batches of 383 and 363
// dipolar stars of 20 and 21 spins (8 sweeps per step against 4: 29.2
// against 30.0 and 57.8 against 62.2 ms per step); with 0.5 the model picks
// 13, the fastest width, in all eight cases.
constexpr int kModelSMs = 152;  // SMs of the GB300 the model was measured on
constexpr double kPipeSweepCost = 0.5;
static int make_plan(const spinrp_system &s, int prec, Plan *plan, int njobs = 1) {
  std::string err;
  const int c = low_bits(prec);
  if (s.tileK[prec] || prec != SPINRP_C64) {
    const int K = std::min(s.tileK[prec] ? s.tileK[prec] : c128_tile(s.M), s.M);
    if (!build_plan(s.M, s.bonds, K, c, plan, &err)) return fail(SPINRP_EINVAL, "%s", err.c_str());
    return SPINRP_OK;
  }
  if (s.M <= 12) {
    if (!build_plan(s.M, s.bonds, s.M, c, plan, &err)) return fail(SPINRP_EINVAL, "%s", err.c_str());
    return SPINRP_OK;
  }
  const double share = std::ldexp((double)njobs, s.M) / kModelSMs;
  bool have = false;
  double best = 0.0;
  for (int K : {13, 12, 14}) {
    if (K > s.M) continue;
    Plan p;
    if (!build_plan(s.M, s.bonds, K, c, &p, &err)) continue;
    double cost = p.sweeps_per_step() * std::max(std::ldexp(1.0, K), share);
    // the pipelined sweep (pipe_grid's conditions; oriented storage, if asked
    // for, may leave it out)
    const bool pipelined = K == 13 && s.M > 13 && (s.regbits == 0 || s.regbits == 6) && s.orient_mode == 0 &&
                           std::ldexp((double)njobs, s.M - 13) >= 4.0 * kModelSMs;
    if (pipelined) cost *= kPipeSweepCost;
    if (!have || cost < best) best = cost, *plan = std::move(p), have = true;
  }
  if (!have) return fail(SPINRP_EINVAL, "%s", err.c_str());
  return SPINRP_OK;
}

extern "C" int spinrp_system_plan_info(const spinrp_system *sys, int prec, int *segments,
                                       int *sweeps_per_step, int *K) {
  if (!sys || (prec != SPINRP_C64 && prec != SPINRP_C128))
    return fail(SPINRP_EINVAL, "system_plan_info: bad argument");
  Plan p;
  int rc = make_plan(*sys, prec, &p);
  if (rc) return rc;
  if (segments) *segments = p.segments();
  if (sweeps_per_step) *sweeps_per_step = p.sweeps_per_step();
  if (K) *K = p.K;
  return SPINRP_OK;
}

extern "C" int spinrp_system_plan_gates(const spinrp_system *sys, int prec, int32_t *pairs,
                                        int32_t *segment, int cap, int *n) {
  if (!sys || !n || (prec != SPINRP_C64 && prec != SPINRP_C128) || (cap > 0 && (!pairs || !segment)))
    return fail(SPINRP_EINVAL, "system_plan_gates: bad argument");
  Plan p;
  int rc = make_plan(*sys, prec, &p);
  if (rc) return rc;
  int k = 0;
  for (int sgi = 0; sgi < p.segments(); ++sgi)
    for (const PlanGate &g : p.seg[sgi]) {
      if (k < cap) pairs[2 * k] = g.i + 1, pairs[2 * k + 1] = g.j + 1, segment[k] = sgi;
      ++k;
    }
  *n = k;
  return SPINRP_OK;
}

// ---------------------------------------------------------------------------
// states
// ---------------------------------------------------------------------------
namespace {

constexpr int64_t kStage = 1 << 16;  // amplitudes per host<->device staging chunk

struct PassSet {
  // sweep descriptors (host copies) and their op lists
  std::vector<PassDesc> desc;
  std::vector<Op> ops;
  // register-blocked programs
  std::vector<PhaseDesc> phases;
  std::vector<ROp> rops;
  // launch roles (indices into desc)
  int head = -1, mid = -1, join = -1, tail = -1;
  std::vector<int> body, bodyr;
  int only = -1, first = -1, midstep = -1, last = -1;
  bool phased = false;  // the register-blocked programs are in use
  int rb = 5;           // their register bits per phase
  bool oriented = false;  // the programs are oriented (and so is the state)
  uint64_t black = 0;     // first-colour spins (logical mask) when oriented
};

struct Layout {  // byte offsets inside the work buffer
  size_t series, partials, ticket, job, coefs, bvals, adiag, qdiag, passes, ops, phases, rops, stage,
      stage_idx, psites, site_series, sops, total;
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

struct spinrp_state {
  int M = 0, prec = 0, device = 0;
  cudaStream_t stream = nullptr;
  void *psi = nullptr;
  unsigned char *work = nullptr;
  bool own_psi = false, own_work = false;
  int64_t cap = 0, len = 0;
  bool ready = false;
  bool has_diag = false;
  int nb = 0;
  Plan plan;
  PassSet ps;
  Layout lay{};
  int max_blocks = 0;
  double coef_dt = NAN;
  std::vector<double> bvals, a;
  std::vector<uint8_t> logical_of;  // physical position -> logical spin
  // device views
  double *series = nullptr;
  double2 *partials = nullptr;
  double *psites = nullptr, *site_series = nullptr;
  bool sites_req = false;     // all-site readout requested for the next init / load
  bool sites = false;         // all-site readout active for the current series
  unsigned *ticket = nullptr;
  GateCoef *coefs = nullptr;
  double *d_bvals = nullptr, *d_a = nullptr;
  uint64_t *qdiag = nullptr;
  PassDesc *passes = nullptr;
  Op *ops = nullptr;
  PhaseDesc *phases = nullptr;
  ROp *rops = nullptr;
  bool v2 = false;
  double2 *stage = nullptr;
  int64_t *stage_idx = nullptr;
  JobPtrs *d_job = nullptr;   // this state's pointer table (one job)
  JobPtrs hjob{};             // the same, host copy (passed with each sweep launch)
  unsigned prefetch_ahead = 0;  // L2 prefetch distance of the register-blocked sweep
  unsigned pipe_blocks = 0;   // blocks of the pipelined sweep, 0 when the plan does not take it
  bool pipe_req = true;       // pipelined sweeps where the plan takes them
  uint64_t orient_black = 0;  // oriented state: first-colour spins (logical), else 0
  uint64_t orient_phys = 0;   // the same as physical positions of the step-boundary layout
  int64_t *d_step = nullptr;  // device series counter
  // CUDA graphs of kGraphSteps steady-state Trotter steps (captured on first use)
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graphs[2] = {nullptr, nullptr};
  // measurement
  bool prof = false;
  std::vector<cudaEvent_t> ev[3];  // start/stop pairs per kernel kind
  int64_t h2d = 0, d2h = 0;
};

// Bracket a launch of kernel kind `kind` with events when profiling is on.
static void prof_mark(spinrp_state *st, int kind) {
  if (!st->prof) return;
  cudaEvent_t e;
  if (cudaEventCreate(&e) == cudaSuccess) {
    cudaEventRecord(e, st->stream);
    st->ev[kind].push_back(e);
  }
}

static void prof_clear(spinrp_state *st) {
  for (auto &v : st->ev) {
    for (cudaEvent_t e : v) cudaEventDestroy(e);
    v.clear();
  }
}

static int init_blocks(int M) {
  const int64_t n = (int64_t(1) << M) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(n, 152 * 8));
}

// Build the sweep descriptors for plan p.
static void build_passes(const Plan &p, bool has_diag, PassSet *ps) {
  const int M = p.M, K = p.K, c = p.c;
  ps->desc.clear();
  ps->ops.clear();
  std::vector<std::vector<int>> pass_in;  // read layout (logical -> physical) of each pass
  // A pass over segment seg that reads the state in layout Lin and writes it in
  // layout Lout (Lout permutes the tile's spins among the tile's positions).
  auto new_pass = [&](int seg, const std::vector<int> &Lin, const std::vector<int> &Lout) -> int {
    PassDesc d;
    memset(&d, 0, sizeof d);
    d.K = K;
    std::vector<int> tpos;
    for (int q : p.segQ[seg]) tpos.push_back(Lin[q]);
    std::sort(tpos.begin(), tpos.end());
    std::vector<char> in(M, 0);
    for (int x : tpos) in[x] = 1;
    int no = 0;
    for (int x = 0; x < M; ++x)
      if (!in[x]) d.outer_pos[no++] = (uint8_t)x;
    std::vector<int> in_spin(M, -1), out_spin(M, -1);  // physical position -> spin
    for (int q = 0; q < M; ++q) in_spin[Lin[q]] = q, out_spin[Lout[q]] = q;
    d.relabel = 0;
    for (int qo = 0; qo < K; ++qo) {
      d.tile_pos[qo] = (uint8_t)tpos[qo];
      const int spin = out_spin[tpos[qo]];
      int qi = 0;
      while (tpos[qi] != Lin[spin]) ++qi;
      d.perm[qo] = (uint8_t)qi;
      if (qi != qo) d.relabel = 1;
    }
    for (int qo = 0; qo < K; ++qo) d.tile_spin[qo] = (uint8_t)in_spin[tpos[qo]];
    for (int o = 0; o < no; ++o) d.outer_spin[o] = (uint8_t)in_spin[d.outer_pos[o]];
    d.site_pos = Lin[0];
    d.site_tile = -1;
    for (int q = 0; q < K; ++q)
      if (tpos[q] == Lin[0]) d.site_tile = q;
    for (int i = 0; i + 1 < K; ++i) d.store_bit[i] = (uint8_t)(i + 1);
    d.op0 = (int)ps->ops.size();
    d.nops = 0;
    ps->desc.push_back(d);
    pass_in.push_back(Lin);
    return (int)ps->desc.size() - 1;
  };
  auto tile_bit = [&](int pass, int logical) -> int {
    const PassDesc &d = ps->desc[pass];
    for (int q = 0; q < K; ++q)
      if (d.tile_pos[q] == pass_in[pass][logical]) return q;
    return -1;
  };
  auto push = [&](int pass, Op op) {
    ps->ops.push_back(op);
    ps->desc[pass].nops++;
  };
  auto gate = [&](int pass, const PlanGate &g, int variant) {
    Op op{};
    op.kind = OP_GATE;
    op.u = (uint8_t)tile_bit(pass, g.i);
    op.v = (uint8_t)tile_bit(pass, g.j);
    op.coef = 2 * g.bond + variant;
    push(pass, op);
  };
  auto diag = [&](int pass, int variant) {
    if (!has_diag) return;
    Op op{};
    op.kind = OP_DIAG;
    op.arg = (uint8_t)variant;
    push(pass, op);
  };
  auto reduce = [&](int pass) {
    Op op{};
    op.kind = OP_REDUCE;
    push(pass, op);
    ps->desc[pass].has_reduce = 1;
  };
  auto fwd = [&](int pass, int seg) {
    for (const PlanGate &g : p.seg[seg]) gate(pass, g, 0);
  };
  auto rev = [&](int pass, int seg) {
    for (auto it = p.seg[seg].rbegin(); it != p.seg[seg].rend(); ++it) gate(pass, *it, 0);
  };
  // forward then reverse of one segment, the two middle copies of its last gate merged
  auto fwd_rev = [&](int pass, int seg) {
    const auto &g = p.seg[seg];
    const int n = (int)g.size();
    for (int k = 0; k + 1 < n; ++k) gate(pass, g[k], 0);
    if (n > 0) gate(pass, g[n - 1], 1);
    for (int k = n - 2; k >= 0; --k) gate(pass, g[k], 0);
  };
  const std::vector<int> &L0 = p.pos;
  const int s = p.segments();
  if (s == 1) {
    // a whole Trotter step per sweep
    ps->only = new_pass(0, L0, L0), diag(ps->only, 0), fwd_rev(ps->only, 0), reduce(ps->only), diag(ps->only, 0);
    ps->first = new_pass(0, L0, L0), diag(ps->first, 0), fwd_rev(ps->first, 0), reduce(ps->first), diag(ps->first, 1);
    ps->midstep = new_pass(0, L0, L0), fwd_rev(ps->midstep, 0), reduce(ps->midstep), diag(ps->midstep, 1);
    ps->last = new_pass(0, L0, L0), fwd_rev(ps->last, 0), reduce(ps->last), diag(ps->last, 0);
    return;
  }
  ps->head = new_pass(0, L0, L0), diag(ps->head, 0), fwd(ps->head, 0);
  // ascending body sweeps: segment k reads layout L[k-1], writes L[k] with
  // exit set X_k moved into the low bits
  std::vector<std::vector<int>> L(s);
  L[0] = L0;
  for (int k = 1; k < s - 1; ++k) {
    std::vector<int> out = L[k - 1];
    std::vector<int> spin_at(M);
    for (int q = 0; q < M; ++q) spin_at[out[q]] = q;
    const std::vector<int> &X = p.exitX[k];
    for (int x : X) {
      if (out[x] < c) continue;
      for (int pl = 0; pl < c; ++pl) {
        const int y = spin_at[pl];
        if (std::find(X.begin(), X.end(), y) != X.end()) continue;
        std::swap(out[x], out[y]);
        spin_at[out[x]] = x, spin_at[out[y]] = y;
        break;
      }
    }
    L[k] = out;
    const int id = new_pass(k, L[k - 1], L[k]);
    fwd(id, k);
    ps->body.push_back(id);
  }
  ps->mid = new_pass(s - 1, L[s - 2], L[s - 2]), fwd_rev(ps->mid, s - 1);
  for (int k = s - 2; k >= 1; --k) {
    const int id = new_pass(k, L[k], L[k - 1]);
    rev(id, k);
    ps->bodyr.push_back(id);
  }
  ps->join = new_pass(0, L0, L0), rev(ps->join, 0), reduce(ps->join), diag(ps->join, 1), fwd(ps->join, 0);
  ps->tail = new_pass(0, L0, L0), rev(ps->tail, 0), reduce(ps->tail), diag(ps->tail, 0);
}

static Layout work_layout(int M, int nb, int64_t cap, const PassSet &ps, int max_blocks) {
  const size_t npass = ps.desc.size(), nops = ps.ops.size();
  Layout L{};
  size_t o = 0;
  L.series = o, o = align256(o + sizeof(double) * 2 * std::max<int64_t>(cap, 1));
  L.partials = o, o = align256(o + sizeof(double2) * max_blocks);
  L.ticket = o, o = align256(o + 256);  // ticket at +0, series counter at +64
  L.job = o, o = align256(o + sizeof(JobPtrs));
  L.coefs = o, o = align256(o + sizeof(GateCoef) * 2 * std::max(nb, 1));
  L.bvals = o, o = align256(o + sizeof(double) * std::max(nb, 1));
  L.adiag = o, o = align256(o + sizeof(double) * M * M);
  L.qdiag = o, o = align256(o + sizeof(uint64_t) * 2 * M * M);
  L.passes = o, o = align256(o + sizeof(PassDesc) * std::max<size_t>(npass, 1));
  L.ops = o, o = align256(o + sizeof(Op) * std::max<size_t>(nops, 1));
  L.phases = o, o = align256(o + sizeof(PhaseDesc) * std::max<size_t>(ps.phases.size(), 1));
  L.rops = o, o = align256(o + sizeof(ROp) * std::max<size_t>(ps.rops.size(), 1));
  L.stage = o, o = align256(o + sizeof(double2) * kStage);
  L.stage_idx = o, o = align256(o + sizeof(int64_t) * kStage);
  L.psites = o, o = align256(o + sizeof(double) * (M + 1) * (size_t)max_blocks);
  L.site_series = o, o = align256(o + sizeof(double) * M * (size_t)std::max<int64_t>(cap, 1));
  L.sops = o, o = align256(o + sizeof(ROpRes) * std::max<size_t>(ps.rops.size(), 1));
  L.total = o;
  return L;
}

// Register-blocked tiles are used when the tile has at least 5 lane bits
// besides the rb register bits (2^(K-rb) threads); complex128 runs five
// register bits (32 FP64 amplitudes per thread).
static bool use_phases(int prec, int K, int rb) {
  return prec == SPINRP_C64 ? K >= 5 + rb : (rb == 5 && K >= 10);
}
// Six register bits (fewer phases, so fewer shared-memory round trips per
// gate) on tiles of 13 and 14 spins; five on narrower tiles, where twice the
// threads per tile measured faster (GB300, ladders and stars of 14..24 spins).
static int default_regbits(int K) { return K >= 13 ? 6 : 5; }

// Compile every pass into phases of RB register bits: the pass's gates
// between two element-wise ops (diagonal phase, reduction) are cut into
// phases by the same greedy as the sweep planner (gates on disjoint bits may
// be exchanged, nothing else), and each element-wise op runs in the phase
// after the gates it follows.
constexpr int kPhaseBeam = 8;  // beam width of the phase planner

static bool compile_phases(PassSet *ps, int M, int K, int RB, int prec, std::string *err,
                           bool oriented = false, uint64_t black = 0) {
  ps->phases.clear();
  ps->rops.clear();
  const bool wide = prec != SPINRP_C64;  // 16-byte amplitudes, swizzle_slot16
  auto slot_of = [&](uint32_t t) { return wide ? swizzle_slot16(t) : swizzle_slot(t); };
  // lane bits of distinct residues mod `nres` give an access group distinct
  // banks: four (mod 4) for 8-byte amplitudes, three (mod 3) for 16-byte ones
  const int nres = wide ? 3 : 4;
  for (PassDesc &d : ps->desc) {
    // store order: chunk-index bits 0..2 are output bits 1..3 (128-byte runs);
    // the fourth, the last lane bit of a half-warp, is the output bit whose
    // input bit completes four distinct slot residues, so the half-warp's
    // 8-byte gathers from the tile hit 16 distinct bank pairs
    {
      auto nib = [&](int q) { return swizzle_slot(1u << d.perm[q]) & 15u; };
      std::vector<int> order = {1, 2, 3};
      int pick = -1;
      for (int x = 4; x < K && pick < 0; ++x) {
        const uint32_t a = nib(1), b = nib(2), c = nib(3), e = nib(x);
        // independence of the four nibbles over GF(2)
        bool indep = true;
        for (int m = 1; m < 16 && indep; ++m) {
          const uint32_t v = ((m & 1) ? a : 0u) ^ ((m & 2) ? b : 0u) ^ ((m & 4) ? c : 0u) ^ ((m & 8) ? e : 0u);
          if (v == 0u) indep = false;
        }
        if (indep) pick = x;
      }
      if (K >= 5) {
        if (pick < 0) pick = 4;
        order.push_back(pick);
        for (int x = 4; x < K; ++x)
          if (x != pick) order.push_back(x);
        for (int i = 0; i + 1 < K; ++i) d.store_bit[i] = (uint8_t)order[i];
      }
    }
    d.phase0 = (int)ps->phases.size();
    d.nphases = 0;
    d.rop0 = (int)ps->rops.size();
    // oriented: the tile bits and outer positions of first-colour spins
    d.black_tile = 0;
    d.black_outer = 0;
    if (oriented) {
      for (int q = 0; q < K; ++q)
        if ((black >> d.tile_spin[q]) & 1ull) d.black_tile |= 1u << q;
      for (int o = 0; o < M - K; ++o)
        if ((black >> d.outer_spin[o]) & 1ull) d.black_outer |= 1ull << d.outer_pos[o];
    }
    std::vector<int> default_rb(RB);
    for (int k = 0; k < RB; ++k) default_rb[k] = k;
    std::vector<ROp> pending;  // element-wise ops waiting for the next phase
    auto new_phase = [&](const std::vector<int> &rb) {
      PhaseDesc ph;
      memset(&ph, 0, sizeof ph);
      uint32_t isreg = 0;
      for (int k = 0; k < RB; ++k) ph.rb[k] = (uint8_t)rb[k], isreg |= 1u << rb[k];
      // lane bits: nres non-register bits of distinct residues mod nres
      // (bank-conflict free with the shared-memory swizzle), then the lowest left
      std::vector<int> free_bits, lanes;
      for (int b = 0; b < K; ++b)
        if (!((isreg >> b) & 1)) free_bits.push_back(b);
      uint32_t used = 0, res = 0;
      for (int b : free_bits)
        if ((int)lanes.size() < nres && !((res >> (b % nres)) & 1))
          lanes.push_back(b), used |= 1u << b, res |= 1u << (b % nres);
      for (int b : free_bits)
        if (lanes.size() < 5 && !((used >> b) & 1)) lanes.push_back(b), used |= 1u << b;
      for (int k = 0; k < 5; ++k) ph.lanes[k] = (uint8_t)lanes[k];
      int nw = 0;
      for (int b : free_bits)
        if (!((used >> b) & 1)) ph.warps[nw++] = (uint8_t)b;
      for (int k = 0; k < RB; ++k) ph.sm[k] = (uint16_t)slot_of(1u << ph.rb[k]);
      for (int k = 0; k < 5; ++k) ph.tslot[k] = (uint16_t)slot_of(1u << ph.lanes[k]);
      for (int k = 0; k < K - RB - 5; ++k) ph.tslot[5 + k] = (uint16_t)slot_of(1u << ph.warps[k]);
      ph.op0 = (int)ps->rops.size();
      ph.nops = 0;
      for (const ROp &r : pending) ps->rops.push_back(r), ph.nops++;
      pending.clear();
      ps->phases.push_back(ph);
      d.nphases++;
    };
    auto push_rop = [&](const ROp &r) {
      ps->rops.push_back(r);
      ps->phases.back().nops++;
    };
    bool last_is_diag = false;  // the last phase is a diagonal-only phase
    // an element-wise op (the readout) between gates of one group: gates
    // before it must all be applied first; it runs inside the phase that
    // completes them (each thread reads its own amplitudes, whose gates so far
    // acted within the thread's subcube)
    int fence = -1;
    ROp fence_op{};
    auto flush = [&](std::vector<const Op *> &gates) {
      if (gates.empty()) return true;
      last_is_diag = false;
      std::vector<std::pair<int, int>> pairs;
      for (const Op *g : gates) pairs.push_back({g->u, g->v});
      std::vector<uint32_t> sets;
      std::vector<std::vector<int>> applied;
      const int fz = fence < 0 ? (int)gates.size() : fence;
      int pre_done = 0;
      if (!plan_phases(K, pairs, RB, kPhaseBeam, fz, &sets, &applied, d.black_tile,
                       oriented ? kOrientNbMask(RB) : 0u)) {
        *err = "phase planning failed";
        return false;
      }
      for (size_t k = 0; k < sets.size(); ++k) {
        std::vector<int> rb;
        if (oriented) {
          // the NB first-colour bits first, then the others
          for (int q = 0; q < K; ++q)
            if (((sets[k] >> q) & 1) && ((d.black_tile >> q) & 1)) rb.push_back(q);
          for (int q = 0; q < K; ++q)
            if (((sets[k] >> q) & 1) && !((d.black_tile >> q) & 1)) rb.push_back(q);
        } else {
          for (int q = 0; q < K; ++q)
            if ((sets[k] >> q) & 1) rb.push_back(q);
          // register bit 0 is the pack bit of the complex64 kernel: the bit the
          // fewest of this phase's gates touch (their arithmetic is scalar)
          int pack = 0, best = 1 << 30;
          for (int q = 0; q < (int)rb.size(); ++q) {
            int n = 0;
            for (int gi : applied[k]) n += (pairs[gi].first == rb[q]) + (pairs[gi].second == rb[q]);
            if (n < best) best = n, pack = q;
          }
          std::rotate(rb.begin(), rb.begin() + pack, rb.begin() + pack + 1);
        }
        new_phase(rb);
        const int nbk = oriented ? __builtin_popcount(sets[k] & d.black_tile) : 0;
        ps->phases.back().nb = (uint8_t)nbk;
        for (int gi : applied[k]) {
          const PlanGate g{gi, pairs[gi].first, pairs[gi].second};
          int ku = (int)(std::find(rb.begin(), rb.end(), g.i) - rb.begin());
          int kv = (int)(std::find(rb.begin(), rb.end(), g.j) - rb.begin());
          if (ku > kv) std::swap(ku, kv);
          int combo;
          if (oriented) {
            // one bit of each colour: ku < nb <= kv
            if (!(ku < nbk && kv >= nbk)) {
              *err = "oriented phase: a gate joins two spins of one colour";
              return false;
            }
            combo = 8 * ku + kv;
          } else {
            // combo = index of (ku, kv) among the RB(RB-1)/2 pairs, lexicographic
            int base_idx = 0;
            for (int i = 0; i < ku; ++i) base_idx += RB - 1 - i;
            combo = base_idx + (kv - ku - 1);
          }
          ROp r{};
          r.kind = OP_GATE;
          r.combo = (uint8_t)combo;
          r.coef = gates[g.bond]->coef;
          push_rop(r);
          if (fence >= 0 && gi < fence && ++pre_done == fence) push_rop(fence_op);
        }
      }
      fence = -1;
      gates.clear();
      return true;
    };
    std::vector<const Op *> gates;
    for (int k = 0; k < d.nops; ++k) {
      const Op &op = ps->ops[d.op0 + k];
      if (op.kind == OP_GATE) {
        gates.push_back(&op);
        continue;
      }
      ROp r{};
      r.kind = op.kind;
      r.arg = op.arg;
      if (op.kind == OP_REDUCE && !gates.empty() && fence < 0) {
        fence = (int)gates.size();
        fence_op = r;
        continue;
      }
      if (!flush(gates)) return false;
      if (op.kind == OP_DIAG) {
        // the diagonal phase runs alone (its own phase, no register subcube)
        if (!pending.empty()) new_phase(default_rb);
        pending.push_back(r);
        new_phase(default_rb);
        last_is_diag = true;
      } else if (d.nphases > 0 && pending.empty() && !last_is_diag) {
        push_rop(r);
      } else {
        pending.push_back(r);
      }
    }
    if (!flush(gates)) return false;
    if (!pending.empty() || d.nphases == 0) new_phase(default_rb);
    d.nrops = (int)ps->rops.size() - d.rop0;
    if (d.nphases > kMaxPassPhases || d.nrops > kMaxPassOps) {
      *err = "a sweep's register program exceeds the staging capacity";
      return false;
    }
  }
  return true;
}

// Plans (sweeps, op lists, register programs) depend only on the bond list,
// whether any S^zS^z coupling is present, the precision, the tile and
// register settings and the job count of the tile model; a process-wide cache
// keyed by those serves repeated systems (serving streams, batches, a
// footprint query followed by the state it sizes) without re-planning.
namespace {
struct PlanKey {
  int prec, M, tileK, regbits, njobs;
  bool diag, orient;
  std::vector<std::pair<int, int>> bonds;
  bool operator<(const PlanKey &o) const {
    return std::tie(prec, M, tileK, regbits, njobs, diag, orient, bonds) <
           std::tie(o.prec, o.M, o.tileK, o.regbits, o.njobs, o.diag, o.orient, o.bonds);
  }
};
struct PlanEntry {
  Plan plan;
  PassSet ps;
  int max_blocks;
};
std::mutex g_plan_mu;
std::map<PlanKey, PlanEntry> g_plan_cache;
constexpr size_t kPlanCacheMax = 256;  // entries kept before the cache starts over
}  // namespace

static int plan_state_uncached(const spinrp_system &sys, int prec, Plan *plan, PassSet *ps,
                               int *max_blocks, int njobs, bool orient) {
  int rc = make_plan(sys, prec, plan, njobs);
  if (rc) return rc;
  build_passes(*plan, any_diag(sys), ps);
  ps->phased = false;
  ps->oriented = false;
  ps->black = 0;
  ps->rb = prec != SPINRP_C64 ? 5 : sys.regbits ? sys.regbits : default_regbits(plan->K);
  if (use_phases(prec, plan->K, ps->rb)) {
    // a program too large to stage in shared memory runs the plain kernel;
    // complex64 programs of a 2-colourable system are oriented when every
    // phase can hold its fixed colour pattern, else they are plain
    std::string err;
    if (orient && prec == SPINRP_C64 && sys.bipartite) {
      ps->oriented = compile_phases(ps, sys.M, plan->K, ps->rb, prec, &err, true, sys.black);
      if (ps->oriented) ps->black = sys.black;
    }
    ps->phased = ps->oriented || compile_phases(ps, sys.M, plan->K, ps->rb, prec, &err);
    if (!ps->phased) ps->phases.clear(), ps->rops.clear();
  }
  // every gate on two distinct bits of its tile; every store permutation a permutation
  for (const PassDesc &d : ps->desc) {
    unsigned seen = 0;
    for (int q = 0; q < d.K; ++q) seen |= 1u << d.perm[q];
    if (d.K != plan->K || seen != (1u << d.K) - 1u)
      return fail(SPINRP_EINVAL, "plan: inconsistent store permutation");
    for (int k = 0; k < d.nops; ++k) {
      const Op &op = ps->ops[d.op0 + k];
      if (op.kind == OP_GATE && (op.u >= d.K || op.v >= d.K || op.u == op.v))
        return fail(SPINRP_EINVAL, "plan: gate outside its tile");
    }
  }
  *max_blocks = std::max(init_blocks(sys.M), 1 << (sys.M - plan->K));
  return SPINRP_OK;
}

static int plan_state(const spinrp_system &sys, int prec, Plan *plan, PassSet *ps, int *max_blocks,
                      int njobs = 1, bool allow_orient = true) {
  const bool orient = allow_orient && sys.orient_mode != 0;
  PlanKey key{prec, sys.M, sys.tileK[prec], sys.regbits, njobs, any_diag(sys), orient, sys.bonds};
  {
    std::lock_guard<std::mutex> lock(g_plan_mu);
    auto it = g_plan_cache.find(key);
    if (it != g_plan_cache.end()) {
      *plan = it->second.plan;
      *ps = it->second.ps;
      *max_blocks = it->second.max_blocks;
      return SPINRP_OK;
    }
  }
  const int rc = plan_state_uncached(sys, prec, plan, ps, max_blocks, njobs, orient);
  if (rc) return rc;
  std::lock_guard<std::mutex> lock(g_plan_mu);
  if (g_plan_cache.size() >= kPlanCacheMax) g_plan_cache.clear();
  g_plan_cache.emplace(std::move(key), PlanEntry{*plan, *ps, *max_blocks});
  return SPINRP_OK;
}

extern "C" int spinrp_state_bytes(const spinrp_system *sys, int prec, int64_t series_cap,
                                  size_t *psi_bytes, size_t *work_bytes) {
  if (!sys || (prec != SPINRP_C64 && prec != SPINRP_C128) || series_cap < 1)
    return fail(SPINRP_EINVAL, "state_bytes: bad argument");
  Plan plan;
  PassSet ps;
  int mb = 0;
  int rc = plan_state(*sys, prec, &plan, &ps, &mb);
  if (rc) return rc;
  const size_t amp = prec == SPINRP_C64 ? 8 : 16;
  if (psi_bytes) *psi_bytes = amp << sys->M;
  if (work_bytes)
    *work_bytes = work_layout(sys->M, (int)sys->bonds.size(), series_cap, ps, mb).total;
  return SPINRP_OK;
}

static void free_state(spinrp_state *st) {
  if (!st) return;
  prof_clear(st);
  for (cudaGraphExec_t g : st->graphs)
    if (g) cudaGraphExecDestroy(g);
  if (st->cap_stream) cudaStreamDestroy(st->cap_stream);
  if (st->own_psi && st->psi) cudaFree(st->psi);
  if (st->own_work && st->work) cudaFree(st->work);
  delete st;
}

// Largest dynamic shared memory of resident_kernel: 227 KiB per block less
// its static arrays (diagonal-phase and reduction scratch, under 4 KiB).
constexpr size_t kResidentMaxSmem = size_t(223) * 1024;
constexpr size_t kPipeSmem = size_t(3) << 16;  // pipe_kernel<6, 13, *>: three 64 KiB tile buffers

template <typename R>
static int set_smem_limits() {
  // the widest tile of this precision (2^14 c64 or 2^13 c128 = 128 KiB)
  const int kmax = sizeof(R) == 4 ? 14 : 13;
  const int wide = (int)(sizeof(typename CT<R>::T) << kmax);
  CUDA_TRY(cudaFuncSetAttribute(sweep_kernel<R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, wide));
  CUDA_TRY(cudaFuncSetAttribute(sweep_kernel<R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, wide));
  if (sizeof(R) == 4)
  {
    const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
    CUDA_TRY(cudaFuncSetAttribute(sweep2_kernel<5, false, false>, a, 8 << 14));
    CUDA_TRY(cudaFuncSetAttribute(sweep2_kernel<6, false, false>, a, 8 << 14));
    CUDA_TRY(cudaFuncSetAttribute(sweep2_kernel<5, true, false>, a, 8 << 14));
    CUDA_TRY(cudaFuncSetAttribute(sweep2_kernel<6, true, false>, a, 8 << 14));
    CUDA_TRY(cudaFuncSetAttribute(sweep2_kernel<5, false, true>, a, 8 << 14));
    CUDA_TRY(cudaFuncSetAttribute(sweep2_kernel<6, false, true>, a, 8 << 14));
    CUDA_TRY(cudaFuncSetAttribute(sweep2_kernel<5, true, true>, a, 8 << 14));
    CUDA_TRY(cudaFuncSetAttribute(sweep2_kernel<6, true, true>, a, 8 << 14));
    CUDA_TRY(cudaFuncSetAttribute(pipe_kernel<6, 13, false>, a, (int)kPipeSmem));
    CUDA_TRY(cudaFuncSetAttribute(pipe_kernel<6, 13, true>, a, (int)kPipeSmem));
    CUDA_TRY(cudaFuncSetAttribute(resident_kernel<5, false>, a, (int)kResidentMaxSmem));
    CUDA_TRY(cudaFuncSetAttribute(resident_kernel<5, true>, a, (int)kResidentMaxSmem));
    CUDA_TRY(cudaFuncSetAttribute(resident_kernel<6, false>, a, (int)kResidentMaxSmem));
    CUDA_TRY(cudaFuncSetAttribute(resident_kernel<6, true>, a, (int)kResidentMaxSmem));
  } else {
    CUDA_TRY(cudaFuncSetAttribute(sweep2d_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 16 << 13));
  }
  return SPINRP_OK;
}

// Register-blocked sweep blocks resident on the whole device at once (the L2
// prefetch distance); 0 when the query fails.
static unsigned sweep2_resident(int prec, int rb, int K, bool oriented) {
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const size_t smem = (prec == SPINRP_C64 ? size_t(8) : size_t(16)) << K;
  const cudaError_t e =
      prec != SPINRP_C64
          ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, sweep2d_kernel, 1 << (K - 5), smem)
      : rb == 6 ? (oriented ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, sweep2_kernel<6, false, true>,
                                                                            1 << (K - 6), smem)
                            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, sweep2_kernel<6, false, false>,
                                                                            1 << (K - 6), smem))
                : (oriented ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, sweep2_kernel<5, false, true>,
                                                                            1 << (K - 5), smem)
                            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, sweep2_kernel<5, false, false>,
                                                                            1 << (K - 5), smem));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return (unsigned)(per * sms);
}

// Blocks of the pipelined sweep (pipe_kernel, one per SM) for the plan of
// njobs jobs (a state: 1), or 0 when the plan does not take it: complex64,
// register-blocked with six register bits and 13-spin tiles, more than one
// tile per job, plain storage, and at least four units (tiles of all jobs)
// per SM so that the three-buffer pipeline fills.
static unsigned pipe_grid(int prec, const Plan &plan, const PassSet &ps, int M, int njobs = 1) {
  if (prec != SPINRP_C64 || !ps.phased || ps.rb != 6 || plan.K != 13 || M <= 13 || ps.oriented) return 0;
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, pipe_kernel<6, 13, false>, kPipeThreads, kPipeSmem) !=
          cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const unsigned long long units = (unsigned long long)njobs << (M - 13);
  if (per < 1 || units < 4ull * (unsigned long long)sms || units >= (1ull << 32)) return 0;
  if (njobs > 1)
    for (const PassDesc &pd : ps.desc)
      if (pd.nrops > kPipeBatchOps) return 0;  // a pass's ops must fit a buffer's slice
  return (unsigned)sms;
}

// The state's error word of the pipelined sweep: 128 bytes into the 256-byte
// ticket area (ticket at +0, series counter at +64), cleared with it.
static int *pipe_err_word(spinrp_state *st) {
  return reinterpret_cast<int *>(reinterpret_cast<unsigned char *>(st->ticket) + 128);
}

extern "C" int spinrp_state_create(const spinrp_system *sys, int prec, void *stream,
                                   int64_t series_cap, void *psi, void *work, spinrp_state **out) {
  if (!out) return fail(SPINRP_EINVAL, "state_create: out is NULL");
  *out = nullptr;
  if (!sys || (prec != SPINRP_C64 && prec != SPINRP_C128) || series_cap < 1)
    return fail(SPINRP_EINVAL, "state_create: bad argument");
  if (((uintptr_t)psi & 255) || ((uintptr_t)work & 255))
    return fail(SPINRP_EINVAL, "state_create: buffers must be 256-byte aligned");
  spinrp_state *st = new (std::nothrow) spinrp_state;
  if (!st) return fail(SPINRP_ENOMEM, "state_create: out of host memory");
  st->M = sys->M;
  st->prec = prec;
  st->stream = (cudaStream_t)stream;
  st->cap = series_cap;
  st->nb = (int)sys->bonds.size();
  st->has_diag = any_diag(*sys);
  int rc = plan_state(*sys, prec, &st->plan, &st->ps, &st->max_blocks);
  if (rc) {
    delete st;
    return rc;
  }
  st->lay = work_layout(st->M, st->nb, series_cap, st->ps, st->max_blocks);
  for (auto &bd : sys->bonds) st->bvals.push_back(sys->b[bd.first * sys->M + bd.second]);
  st->a = sys->a;
  st->logical_of.assign(st->M, 0);
  for (int q = 0; q < st->M; ++q) st->logical_of[st->plan.pos[q]] = (uint8_t)q;

  cudaError_t e = cudaGetDevice(&st->device);
  if (e != cudaSuccess) {
    delete st;
    return fail(SPINRP_ECUDA, "state_create: cudaGetDevice: %s", cudaGetErrorString(e));
  }
  const size_t psi_bytes = (prec == SPINRP_C64 ? size_t(8) : size_t(16)) << st->M;
  if (psi) {
    st->psi = psi;
  } else {
    e = cudaMalloc(&st->psi, psi_bytes);
    if (e != cudaSuccess) {
      delete st;
      cudaGetLastError();
      return fail(SPINRP_ENOMEM, "state_create: cudaMalloc(%zu): %s", psi_bytes, cudaGetErrorString(e));
    }
    st->own_psi = true;
  }
  if (work) {
    st->work = (unsigned char *)work;
  } else {
    e = cudaMalloc((void **)&st->work, st->lay.total);
    if (e != cudaSuccess) {
      free_state(st);
      cudaGetLastError();
      return fail(SPINRP_ENOMEM, "state_create: cudaMalloc(%zu): %s", st->lay.total, cudaGetErrorString(e));
    }
    st->own_work = true;
  }
  unsigned char *w = st->work;
  st->series = (double *)(w + st->lay.series);
  st->partials = (double2 *)(w + st->lay.partials);
  st->ticket = (unsigned *)(w + st->lay.ticket);
  st->coefs = (GateCoef *)(w + st->lay.coefs);
  st->d_bvals = (double *)(w + st->lay.bvals);
  st->d_a = (double *)(w + st->lay.adiag);
  st->qdiag = (uint64_t *)(w + st->lay.qdiag);
  st->passes = (PassDesc *)(w + st->lay.passes);
  st->ops = (Op *)(w + st->lay.ops);
  st->phases = (PhaseDesc *)(w + st->lay.phases);
  st->rops = (ROp *)(w + st->lay.rops);
  st->v2 = st->ps.phased;
  st->stage = (double2 *)(w + st->lay.stage);
  st->stage_idx = (int64_t *)(w + st->lay.stage_idx);
  st->psites = (double *)(w + st->lay.psites);
  st->site_series = (double *)(w + st->lay.site_series);
  st->d_step = (int64_t *)(w + st->lay.ticket + 64);
  st->d_job = (JobPtrs *)(w + st->lay.job);
  JobPtrs hj{};
  hj.psi = st->psi;
  hj.coefs = st->coefs;
  hj.qdiag = st->qdiag;
  hj.partials = st->partials;
  hj.ticket = st->ticket;
  hj.step = st->d_step;
  hj.series = st->series;
  hj.bvals = st->d_bvals;
  hj.a = st->d_a;
  hj.psites = st->psites;
  hj.site_series = st->site_series;
  hj.sops = (ROpRes *)(w + st->lay.sops);
  st->hjob = hj;

  auto up = [&](void *dst, const void *src, size_t n) -> cudaError_t {
    if (n == 0) return cudaSuccess;
    st->h2d += (int64_t)n;
    return cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, st->stream);
  };
  if ((e = cudaMemsetAsync(st->ticket, 0, 256, st->stream)) != cudaSuccess ||
      (e = up(st->d_job, &hj, sizeof hj)) != cudaSuccess ||
      (e = up(st->d_bvals, st->bvals.data(), sizeof(double) * st->bvals.size())) != cudaSuccess ||
      (e = up(st->d_a, st->a.data(), sizeof(double) * st->a.size())) != cudaSuccess ||
      (e = up(st->passes, st->ps.desc.data(), sizeof(PassDesc) * st->ps.desc.size())) != cudaSuccess ||
      (e = up(st->ops, st->ps.ops.data(), sizeof(Op) * st->ps.ops.size())) != cudaSuccess ||
      (e = up(st->phases, st->ps.phases.data(), sizeof(PhaseDesc) * st->ps.phases.size())) != cudaSuccess ||
      (e = up(st->rops, st->ps.rops.data(), sizeof(ROp) * st->ps.rops.size())) != cudaSuccess ||
      (e = cudaStreamSynchronize(st->stream)) != cudaSuccess) {
    free_state(st);
    return fail(SPINRP_ECUDA, "state_create: upload: %s", cudaGetErrorString(e));
  }
  rc = prec == SPINRP_C64 ? set_smem_limits<float>() : set_smem_limits<double>();
  if (rc) {
    free_state(st);
    return rc;
  }
  if (st->ps.phased) st->prefetch_ahead = sweep2_resident(prec, st->ps.rb, st->plan.K, st->ps.oriented);
  st->pipe_blocks = pipe_grid(prec, st->plan, st->ps, st->M);
  if (st->ps.oriented) {
    st->orient_black = st->ps.black;
    for (int q = 0; q < st->M; ++q)
      if ((st->orient_black >> q) & 1ull) st->orient_phys |= 1ull << st->plan.pos[q];
  }
  *out = st;
  return SPINRP_OK;
}

extern "C" void spinrp_state_destroy(spinrp_state *st) {
  if (!st) return;
  cudaStreamSynchronize(st->stream);
  free_state(st);
}

static LayoutArg layout_arg(const spinrp_state *st) {
  LayoutArg la;
  memset(&la, 0, sizeof la);
  for (int p = 0; p < st->M; ++p) la.logical_of[p] = st->logical_of[p];
  return la;
}

// Apply the requested readout mode at the start of a series; cached graphs
// hold the launches of the previous mode and are dropped when it changes.
static void begin_series(spinrp_state *st) {
  if (st->sites != st->sites_req) {
    for (cudaGraphExec_t &g : st->graphs)
      if (g) cudaGraphExecDestroy(g), g = nullptr;
    st->sites = st->sites_req;
  }
}

// All-site entry 0 (after init / load recorded entry 0 of the main series).
static int record_sites0(spinrp_state *st) {
  if (!st->sites) return SPINRP_OK;
  const int blocks = init_blocks(st->M);
  g_launches += 2;
  if (st->prec == SPINRP_C64)
    state_sites_kernel<float><<<blocks, 256, 0, st->stream>>>(st->d_job, st->M, layout_arg(st));
  else
    state_sites_kernel<double><<<blocks, 256, 0, st->stream>>>(st->d_job, st->M, layout_arg(st));
  CUDA_TRY(cudaGetLastError());
  sites_finalize_kernel<<<st->M, 256, 0, st->stream>>>(st->d_job, st->M, blocks);
  CUDA_TRY(cudaGetLastError());
  return SPINRP_OK;
}

static int state_init(spinrp_state *st, uint64_t seed, int kind) {
  if (!st) return fail(SPINRP_EINVAL, "init: state is NULL");
  begin_series(st);
  const int blocks = init_blocks(st->M);
  prof_mark(st, SPINRP_KERNEL_INIT);
  ++g_launches;
  if (st->prec == SPINRP_C64)
    init_kernel<float><<<blocks, 256, 0, st->stream>>>(st->d_job, st->M, layout_arg(st), seed, nullptr,
                                                       kind, st->orient_black);
  else
    init_kernel<double><<<blocks, 256, 0, st->stream>>>(st->d_job, st->M, layout_arg(st), seed, nullptr,
                                                        kind, st->orient_black);
  CUDA_TRY(cudaGetLastError());
  int rc = record_sites0(st);
  if (rc) return rc;
  prof_mark(st, SPINRP_KERNEL_INIT);
  st->len = 1;
  st->ready = true;
  return SPINRP_OK;
}

extern "C" int spinrp_state_init_random_phase(spinrp_state *st, uint64_t seed) {
  return state_init(st, seed, INIT_ENTANGLED);
}

extern "C" int spinrp_state_init_product_phase(spinrp_state *st, uint64_t seed) {
  return state_init(st, seed, INIT_PRODUCT);
}

// physical index of logical basis index x
static int64_t to_physical(const spinrp_state *st, int64_t x) {
  int64_t y = 0;
  for (int q = 0; q < st->M; ++q) y |= ((x >> q) & 1) << st->plan.pos[q];
  return y;
}

extern "C" int spinrp_state_load(spinrp_state *st, const double *amps) {
  if (!st || !amps) return fail(SPINRP_EINVAL, "load: bad argument");
  begin_series(st);
  const int64_t N = int64_t(1) << st->M;
  std::vector<int64_t> idx;
  for (int64_t k0 = 0; k0 < N; k0 += kStage) {
    const int64_t n = std::min(kStage, N - k0);
    idx.resize(n);
    for (int64_t k = 0; k < n; ++k) idx[k] = to_physical(st, k0 + k);
    CUDA_TRY(cudaMemcpyAsync(st->stage_idx, idx.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice, st->stream));
    CUDA_TRY(cudaMemcpyAsync(st->stage, amps + 2 * k0, sizeof(double2) * n, cudaMemcpyHostToDevice, st->stream));
    st->h2d += (int64_t)(sizeof(int64_t) + sizeof(double2)) * n;
    ++g_launches;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 1024);
    if (st->prec == SPINRP_C64)
      scatter_kernel<float><<<blocks, 256, 0, st->stream>>>((float2 *)st->psi, st->stage_idx, n, st->stage,
                                                            st->orient_phys);
    else
      scatter_kernel<double><<<blocks, 256, 0, st->stream>>>((double2 *)st->psi, st->stage_idx, n, st->stage,
                                                             st->orient_phys);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaStreamSynchronize(st->stream));
  }
  const int blocks = init_blocks(st->M);
  ++g_launches;
  if (st->prec == SPINRP_C64)
    observe_kernel<float><<<blocks, 256, 0, st->stream>>>(st->d_job, st->M, st->plan.pos[0]);
  else
    observe_kernel<double><<<blocks, 256, 0, st->stream>>>(st->d_job, st->M, st->plan.pos[0]);
  CUDA_TRY(cudaGetLastError());
  int rc = record_sites0(st);
  if (rc) return rc;
  CUDA_TRY(cudaStreamSynchronize(st->stream));
  st->len = 1;
  st->ready = true;
  return SPINRP_OK;
}

extern "C" int spinrp_state_read(spinrp_state *st, const int64_t *idx, int64_t n, double *out) {
  if (!st || n < 0 || (n > 0 && (!idx || !out))) return fail(SPINRP_EINVAL, "read: bad argument");
  const int64_t N = int64_t(1) << st->M;
  std::vector<int64_t> pidx;
  for (int64_t k0 = 0; k0 < n; k0 += kStage) {
    const int64_t m = std::min(kStage, n - k0);
    pidx.resize(m);
    for (int64_t k = 0; k < m; ++k) {
      if (idx[k0 + k] < 0 || idx[k0 + k] >= N) return fail(SPINRP_EINVAL, "read: index out of range");
      pidx[k] = to_physical(st, idx[k0 + k]);
    }
    CUDA_TRY(cudaMemcpyAsync(st->stage_idx, pidx.data(), sizeof(int64_t) * m, cudaMemcpyHostToDevice, st->stream));
    st->h2d += (int64_t)sizeof(int64_t) * m;
    st->d2h += (int64_t)sizeof(double2) * m;
    ++g_launches;
    const int blocks = (int)std::min<int64_t>((m + 255) / 256, 1024);
    if (st->prec == SPINRP_C64)
      gather_kernel<float><<<blocks, 256, 0, st->stream>>>((const float2 *)st->psi, st->stage_idx, m, st->stage,
                                                           st->orient_phys);
    else
      gather_kernel<double><<<blocks, 256, 0, st->stream>>>((const double2 *)st->psi, st->stage_idx, m,
                                                            st->stage, st->orient_phys);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaMemcpyAsync(out + 2 * k0, st->stage, sizeof(double2) * m, cudaMemcpyDeviceToHost, st->stream));
    CUDA_TRY(cudaStreamSynchronize(st->stream));
  }
  return SPINRP_OK;
}

extern "C" int spinrp_state_orientation(const spinrp_state *st, uint64_t *black) {
  if (!st || !black) return fail(SPINRP_EINVAL, "state_orientation: bad argument");
  *black = st->orient_black;
  return SPINRP_OK;
}

extern "C" int spinrp_state_set_pipeline(spinrp_state *st, int on) {
  if (!st || (on != 0 && on != 1)) return fail(SPINRP_EINVAL, "state_set_pipeline: bad argument");
  if (st->pipe_req != (on != 0)) {
    // cached graphs hold the launches of the other sweep kernel
    for (cudaGraphExec_t &g : st->graphs)
      if (g) cudaGraphExecDestroy(g), g = nullptr;
    st->pipe_req = on != 0;
  }
  return SPINRP_OK;
}

extern "C" int spinrp_state_pipeline(const spinrp_state *st, int *on) {
  if (!st || !on) return fail(SPINRP_EINVAL, "state_pipeline: bad argument");
  *on = (st->pipe_req && st->pipe_blocks > 0) ? 1 : 0;
  return SPINRP_OK;
}

extern "C" int spinrp_state_pipeline_timeout_check(spinrp_state *st, double *seconds) {
  if (!st) return fail(SPINRP_EINVAL, "state_pipeline_timeout_check: state is NULL");
  if (!st->pipe_blocks || st->ps.desc.empty())
    return fail(SPINRP_ESTATE, "state_pipeline_timeout_check: the state's sweeps do not run pipelined");
  int *err = pipe_err_word(st);
  cudaEvent_t e0, e1;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  cudaEventRecord(e0, st->stream);
  // probe = 1: the producer issues no copies, so every wait of every block
  // runs out; nothing is written to the amplitudes or the series
  pipe_kernel<6, 13, false><<<st->pipe_blocks, kPipeThreads, kPipeSmem, st->stream>>>(
      st->d_job, 1, static_cast<float2 *>(st->psi), st->hjob.sops, 0, st->ps.desc[0], st->phases, st->M, err, 1);
  cudaEventRecord(e1, st->stream);
  ++g_launches;
  const cudaError_t le = cudaGetLastError();
  int flag = 0;
  cudaError_t ce = cudaMemcpyAsync(&flag, err, sizeof flag, cudaMemcpyDeviceToHost, st->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st->stream);
  float ms = 0.f;
  if (ce == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (le != cudaSuccess || ce != cudaSuccess)
    return fail(SPINRP_ECUDA, "state_pipeline_timeout_check: %s", cudaGetErrorString(le != cudaSuccess ? le : ce));
  if (seconds) *seconds = ms / 1e3;
  CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), st->stream));
  CUDA_TRY(cudaStreamSynchronize(st->stream));
  return flag ? fail(SPINRP_ETIMEOUT, "state_pipeline_timeout_check: the waits ran out as intended")
              : fail(SPINRP_ECUDA, "state_pipeline_timeout_check: no wait ran out");
}

extern "C" int spinrp_state_layout(const spinrp_state *st, int32_t *layout, void **psi) {
  if (!st) return fail(SPINRP_EINVAL, "layout: state is NULL");
  if (layout)
    for (int q = 0; q < st->M; ++q) layout[q] = st->plan.pos[q];
  if (psi) *psi = st->psi;
  return SPINRP_OK;
}

// What the launch helpers need to run a plan over njobs jobs (a state is a
// plan with one job; a batch has one context per plan group).
struct LaunchCtx {
  int M = 0, K = 0;
  bool v2 = false;
  int segments = 1, sweeps_per_step = 1;
  const PassSet *ps = nullptr;
  const PassDesc *passes = nullptr;
  const Op *ops = nullptr;
  const PhaseDesc *phases = nullptr;
  const ROp *rops = nullptr;
  const JobPtrs *jobs = nullptr;
  JobPtrs job0{};  // host copy of the only job's pointers when njobs == 1
  int njobs = 1;
  int rb = 5;                    // register bits of the register-blocked kernel
  bool oriented = false;         // oriented program and state (complex64)
  int sites = 0;                 // all-site readout after every reducing sweep
  unsigned prefetch_ahead = 0;   // sweep blocks resident at once (L2 prefetch distance), 0 = off
  bool resident = false;         // whole state kept in shared memory for every step (resident_kernel)
  unsigned pipe_blocks = 0;      // > 0: one-job sweeps of the plan run as pipe_kernel on this many blocks
  int *pipe_err = nullptr;       // its error word
  JobPtrs batch0{};              // batch group: the first job's pointers ...
  long long job_stride = 0;      // ... and the byte distance between consecutive jobs' buffers
  size_t resident_smem = 0;      // its dynamic shared memory
  spinrp_state *prof = nullptr;  // state whose profiling marks to record, if any
};

// Dynamic shared memory of resident_kernel for a plan, or 0 when the plan
// cannot run resident: complex64, one tile holding the whole state (one
// segment, register-blocked program), no all-site readout, and the state plus
// the program within the 227 KiB a block may use.
static size_t resident_bytes(const Plan &plan, const PassSet &ps, int prec, bool sites) {
  if (prec != SPINRP_C64 || !ps.phased || plan.segments() != 1 || plan.K != plan.M || sites) return 0;
  if (ps.only < 0 || ps.first < 0 || ps.midstep < 0 || ps.last < 0) return 0;
  if (plan.M - ps.rb > 8) return 0;  // at most 256 threads per block
  const size_t b = (size_t(8) << plan.M) + sizeof(PhaseDesc) * ps.phases.size() +
                   sizeof(ROpRes) * ps.rops.size();
  return b <= kResidentMaxSmem ? b : 0;
}

// All steps of an evolve call of a resident context: one launch.
static int launch_resident(const LaunchCtx &c, cudaStream_t stream, int64_t steps, bool live) {
  ResidentPasses rp;
  rp.first = c.ps->desc[c.ps->first];
  rp.mid = c.ps->desc[c.ps->midstep];
  rp.last = c.ps->desc[c.ps->last];
  rp.only = c.ps->desc[c.ps->only];
  const int nph = (int)c.ps->phases.size(), nrops = (int)c.ps->rops.size();
  const dim3 grid(1, (unsigned)c.njobs);
  const unsigned nt = 1u << (c.M - c.rb);
  if (live) {
    if (c.prof) prof_mark(c.prof, SPINRP_KERNEL_SWEEP);
    ++g_launches;
  }
  const int code = (c.rb == 6 ? 2 : 0) | (c.oriented ? 1 : 0);
#define RES(RB_, O_) \
  resident_kernel<RB_, O_><<<grid, nt, c.resident_smem, stream>>>(c.jobs, rp, c.phases, nph, nrops, c.M, steps)
  switch (code) {
    case 0: RES(5, false); break;
    case 1: RES(5, true); break;
    case 2: RES(6, false); break;
    default: RES(6, true); break;
  }
#undef RES
  CUDA_TRY(cudaGetLastError());
  if (live && c.prof) prof_mark(c.prof, SPINRP_KERNEL_SWEEP);
  return SPINRP_OK;
}

// Launch one sweep on `stream`; `live` launches are counted and profiled,
// launches recorded into a graph are not.
template <typename R>
static int launch_pass(const LaunchCtx &c, int pass, cudaStream_t stream, bool live) {
  const int K = c.K;
  const int nt = std::min(512, std::max(32, 1 << K));
  const size_t smem = sizeof(typename CT<R>::T) << K;
  const dim3 grid(1u << (c.M - K), (unsigned)c.njobs);
  if (live) {
    if (c.prof) prof_mark(c.prof, SPINRP_KERNEL_SWEEP);
    ++g_launches;
  }
  // the all-site sums are taken only in the sweep that reads P out; the
  // other sweeps of an all-site run are the plain ones
  const bool sites = c.sites && c.ps->desc[pass].has_reduce;
  if (sizeof(R) == 4 && c.v2)
  {
    const size_t sm2 = size_t(8) << K;
    const PassDesc &pd = c.ps->desc[pass];
    float2 *psi1 = c.njobs == 1 ? static_cast<float2 *>(c.job0.psi) : nullptr;
    const unsigned ahead = c.prefetch_ahead;
    const ROpRes *sops1 = c.njobs == 1 ? c.job0.sops : nullptr;
    const int code = (c.rb == 6 ? 4 : 0) | (sites ? 2 : 0) | (c.oriented ? 1 : 0);
    const bool piped = c.pipe_blocks && K == 13 && code == 4;
    if (piped) {
      if (c.njobs == 1)
        pipe_kernel<6, 13, false><<<c.pipe_blocks, kPipeThreads, kPipeSmem, stream>>>(
            c.jobs, 1, psi1, sops1, 0, pd, c.phases, c.M, c.pipe_err, 0);
      else
      {
        pipe_kernel<6, 13, true><<<c.pipe_blocks, kPipeThreads, kPipeSmem, stream>>>(
            c.jobs, c.njobs, static_cast<float2 *>(c.batch0.psi), c.batch0.sops, c.job_stride, pd, c.phases, c.M,
            c.pipe_err, 0);
        if (pd.has_reduce) {
          CUDA_TRY(cudaGetLastError());
          if (live) ++g_launches;
          pipe_finalize_kernel<<<c.njobs, 128, 0, stream>>>(c.jobs, 1u << (c.M - 13), c.pipe_err);
        }
      }
    } else {
#define SW2(RB_, S_, O_) \
  sweep2_kernel<RB_, S_, O_><<<grid, 1 << (K - RB_), sm2, stream>>>(c.jobs, psi1, sops1, pd, c.phases, c.M, ahead)
      switch (code) {
        case 0: SW2(5, false, false); break;
        case 1: SW2(5, false, true); break;
        case 2: SW2(5, true, false); break;
        case 3: SW2(5, true, true); break;
        case 4: SW2(6, false, false); break;
        case 5: SW2(6, false, true); break;
        case 6: SW2(6, true, false); break;
        default: SW2(6, true, true); break;
      }
#undef SW2
    }
  }
  else if (sizeof(R) == 8 && c.v2 && !sites)
    // complex128 register-blocked (the all-site sums run in the plain kernel)
    sweep2d_kernel<<<grid, 1 << (K - 5), smem, stream>>>(c.jobs, c.ps->desc[pass], c.phases, c.rops, c.M,
                                                          c.prefetch_ahead);
  else if (sites)
    sweep_kernel<R, true><<<grid, nt, smem, stream>>>(c.jobs, c.passes + pass, c.ops, c.M);
  else
    sweep_kernel<R, false><<<grid, nt, smem, stream>>>(c.jobs, c.passes + pass, c.ops, c.M);
  CUDA_TRY(cudaGetLastError());
  if (c.sites && c.ps->desc[pass].has_reduce) {
    if (live) ++g_launches;
    sites_finalize_kernel<<<dim3(c.M, c.njobs), 256, 0, stream>>>(c.jobs, c.M, 1 << (c.M - K));
    CUDA_TRY(cudaGetLastError());
  }
  if (live && c.prof) prof_mark(c.prof, SPINRP_KERNEL_SWEEP);
  return SPINRP_OK;
}

#define RUN(pass)                                           \
  do {                                                      \
    int rc_ = launch_pass<R>(c, (pass), stream, live);      \
    if (rc_) return rc_;                                    \
  } while (0)

// n steady-state Trotter steps (neither the first nor the last of a call):
// [body, middle, reverse body, join] or, for one segment, [whole step].
template <typename R>
static int steady_steps(const LaunchCtx &c, cudaStream_t stream, int64_t n, bool live) {
  const PassSet &ps = *c.ps;
  for (int64_t k = 0; k < n; ++k) {
    if (c.segments == 1) {
      RUN(ps.midstep);
    } else {
      for (int id : ps.body) RUN(id);
      RUN(ps.mid);
      for (int id : ps.bodyr) RUN(id);
      RUN(ps.join);
    }
  }
  return SPINRP_OK;
}

// First step of an evolve call of `steps` steps (the whole call when steps == 1
// and the plan has one segment).
template <typename R>
static int first_step(const LaunchCtx &c, cudaStream_t stream, int64_t steps, bool live) {
  const PassSet &ps = *c.ps;
  if (c.segments == 1) RUN(steps == 1 ? ps.only : ps.first);
  else RUN(ps.head);
  return SPINRP_OK;
}

template <typename R>
static int last_step(const LaunchCtx &c, cudaStream_t stream, int64_t steps, bool live) {
  const PassSet &ps = *c.ps;
  if (c.segments == 1) {
    if (steps > 1) RUN(ps.last);
  } else {
    for (int id : ps.body) RUN(id);
    RUN(ps.mid);
    for (int id : ps.bodyr) RUN(id);
    RUN(ps.tail);
  }
  return SPINRP_OK;
}
#undef RUN

static int64_t steady_count(const LaunchCtx &c, int64_t steps) {
  return c.segments == 1 ? std::max<int64_t>(0, steps - 2) : steps - 1;
}

constexpr int kGraphSteps = 16;  // steady-state steps per captured CUDA graph

// Capture kGraphSteps steady steps of every context into one graph.
template <typename R>
static int capture_graph(const std::vector<LaunchCtx> &cs, cudaStream_t *cap_stream,
                         cudaGraphExec_t *exec) {
  if (!*cap_stream) CUDA_TRY(cudaStreamCreateWithFlags(cap_stream, cudaStreamNonBlocking));
  CUDA_TRY(cudaStreamBeginCapture(*cap_stream, cudaStreamCaptureModeThreadLocal));
  int rc = SPINRP_OK;
  for (int k = 0; k < kGraphSteps && rc == SPINRP_OK; ++k)
    for (const LaunchCtx &c : cs)
      if (rc == SPINRP_OK) rc = steady_steps<R>(c, *cap_stream, 1, false);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(*cap_stream, &g);
  if (rc != SPINRP_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return rc != SPINRP_OK ? rc : fail(SPINRP_ECUDA, "graph capture: %s", cudaGetErrorString(e));
  }
  const cudaError_t e2 = cudaGraphInstantiate(exec, g, 0);
  cudaGraphDestroy(g);
  if (e2 != cudaSuccess) {
    *exec = nullptr;
    return fail(SPINRP_ECUDA, "graph instantiate: %s", cudaGetErrorString(e2));
  }
  return SPINRP_OK;
}

// `steps` Trotter steps of every context (all share dt and steps): the first
// step, the steady steps (as graph replays when `use_graph`), the last step.
template <typename R>
static int run_steps(const std::vector<LaunchCtx> &all, cudaStream_t stream, int64_t steps,
                     bool use_graph, cudaStream_t *cap_stream, cudaGraphExec_t *graph) {
  // resident contexts run every step in one launch
  std::vector<LaunchCtx> cs;
  for (const LaunchCtx &c : all) {
    if (!c.resident) {
      cs.push_back(c);
      continue;
    }
    int rc = launch_resident(c, stream, steps, true);
    if (rc) return rc;
  }
  for (const LaunchCtx &c : cs) {
    int rc = first_step<R>(c, stream, steps, true);
    if (rc) return rc;
  }
  // every context has the same number of steady steps except single-segment
  // plans (two fewer instead of one); handle them separately
  std::vector<LaunchCtx> multi, single;
  for (const LaunchCtx &c : cs) (c.segments == 1 ? single : multi).push_back(c);
  for (int pass = 0; pass < 2; ++pass) {
    const std::vector<LaunchCtx> &group = pass == 0 ? multi : single;
    if (group.empty()) continue;
    int64_t left = steady_count(group[0], steps);
    cudaGraphExec_t *gexec = graph + pass;
    if (use_graph && left >= kGraphSteps) {
      if (!*gexec) {
        int rc = capture_graph<R>(group, cap_stream, gexec);
        if (rc) return rc;
      }
      int64_t per = 0;
      for (const LaunchCtx &c : group) per += c.segments == 1 ? 1 : c.sweeps_per_step;
      for (; left >= kGraphSteps; left -= kGraphSteps) {
        CUDA_TRY(cudaGraphLaunch(*gexec, stream));
        g_launches += (int64_t)kGraphSteps * per;
      }
    }
    for (int64_t k = 0; k < left; ++k)
      for (const LaunchCtx &c : group) {
        int rc = steady_steps<R>(c, stream, 1, true);
        if (rc) return rc;
      }
  }
  for (const LaunchCtx &c : cs) {
    int rc = last_step<R>(c, stream, steps, true);
    if (rc) return rc;
  }
  return SPINRP_OK;
}

static LaunchCtx state_ctx(spinrp_state *st) {
  LaunchCtx c;
  c.M = st->M;
  c.K = st->plan.K;
  c.v2 = st->v2;
  c.rb = st->ps.rb;
  c.oriented = st->ps.oriented;
  c.sites = st->sites ? 1 : 0;
  c.resident_smem = resident_bytes(st->plan, st->ps, st->prec, st->sites);
  c.resident = c.resident_smem > 0;
  c.prefetch_ahead = st->prefetch_ahead;
  c.pipe_blocks = st->pipe_req ? st->pipe_blocks : 0;
  c.pipe_err = pipe_err_word(st);
  c.segments = st->plan.segments();
  c.sweeps_per_step = st->plan.sweeps_per_step();
  c.ps = &st->ps;
  c.passes = st->passes;
  c.ops = st->ops;
  c.phases = st->phases;
  c.rops = st->rops;
  c.jobs = st->d_job;
  c.job0 = st->hjob;
  c.njobs = 1;
  c.prof = st;
  return c;
}

template <typename R>
static int run_evolve(spinrp_state *st, int64_t steps) {
  return run_steps<R>({state_ctx(st)}, st->stream, steps, !st->prof, &st->cap_stream, st->graphs);
}

extern "C" int spinrp_evolve(spinrp_state *st, double dt, int64_t steps, int order) {
  if (!st) return fail(SPINRP_EINVAL, "evolve: state is NULL");
  if (order != 2) return fail(SPINRP_EUNSUPPORTED, "evolve: only order 2 is implemented");
  if (!st->ready) return fail(SPINRP_ESTATE, "evolve: state not initialized");
  if (!std::isfinite(dt)) return fail(SPINRP_EINVAL, "evolve: dt not finite");
  if (steps < 0) return fail(SPINRP_EINVAL, "evolve: negative steps");
  if (steps == 0) return SPINRP_OK;
  if (st->len + steps > st->cap)
    return fail(SPINRP_EINVAL, "evolve: series capacity %lld exceeded", (long long)st->cap);
  if (!(dt == st->coef_dt)) {
    prof_mark(st, SPINRP_KERNEL_TABLES);
    if (st->nb > 0) {
      ++g_launches;
      coef_kernel<<<(2 * st->nb + 127) / 128, 128, 0, st->stream>>>(st->d_job, st->nb, dt);
      CUDA_TRY(cudaGetLastError());
    }
    if (st->v2 && st->prec == SPINRP_C64 && !st->ps.rops.empty()) {
      const int nr = (int)st->ps.rops.size();
      ++g_launches;
      resolve_ops_kernel<<<(nr + 127) / 128, 128, 0, st->stream>>>(st->d_job, st->rops, nr);
      CUDA_TRY(cudaGetLastError());
    }
    if (st->has_diag) {
      const int n = 2 * st->M * st->M;
      ++g_launches;
      diag_kernel<<<(n + 127) / 128, 128, 0, st->stream>>>(st->d_job, layout_arg(st), st->M, dt);
      CUDA_TRY(cudaGetLastError());
    }
    prof_mark(st, SPINRP_KERNEL_TABLES);
    st->coef_dt = dt;
  }
  int rc = st->prec == SPINRP_C64 ? run_evolve<float>(st, steps) : run_evolve<double>(st, steps);
  if (rc) return rc;
  st->len += steps;
  return SPINRP_OK;
}

extern "C" int64_t spinrp_series_length(const spinrp_state *st) { return st ? st->len : 0; }

static int copy_series(spinrp_state *st, int which, double *out, int64_t cap, int64_t *n) {
  if (!st || !n || (cap > 0 && !out)) return fail(SPINRP_EINVAL, "series: bad argument");
  *n = st->len;
  const int64_t m = std::min(cap, st->len);
  if (m <= 0) return SPINRP_OK;
  std::vector<double> buf(2 * m);
  CUDA_TRY(cudaMemcpyAsync(buf.data(), st->series, sizeof(double) * 2 * m, cudaMemcpyDeviceToHost, st->stream));
  st->d2h += (int64_t)sizeof(double) * 2 * m;
  // a pipelined sweep whose wait gave up recorded NaN and set the error word
  int perr = 0;
  if (st->pipe_blocks) {
    CUDA_TRY(cudaMemcpyAsync(&perr, pipe_err_word(st), sizeof perr, cudaMemcpyDeviceToHost, st->stream));
    st->d2h += (int64_t)sizeof perr;
  }
  CUDA_TRY(cudaStreamSynchronize(st->stream));
  for (int64_t k = 0; k < m; ++k) out[k] = buf[2 * k + which];
  if (perr) return fail(SPINRP_ETIMEOUT, "series: a wait of the pipelined sweep gave up");
  return SPINRP_OK;
}

extern "C" int spinrp_state_set_sites(spinrp_state *st, int all_sites) {
  if (!st) return fail(SPINRP_EINVAL, "set_sites: state is NULL");
  st->sites_req = all_sites != 0;
  return SPINRP_OK;
}

extern "C" int spinrp_site_series(spinrp_state *st, double *out, int64_t cap, int64_t *n) {
  if (!st || !n || (cap > 0 && !out)) return fail(SPINRP_EINVAL, "site_series: bad argument");
  if (!st->ready || !st->sites)
    return fail(SPINRP_ESTATE, "site_series: all-site readout was not enabled at the last init / load");
  *n = st->len;
  const int64_t m = std::min(cap, st->len);
  if (m <= 0) return SPINRP_OK;
  CUDA_TRY(cudaMemcpyAsync(out, st->site_series, sizeof(double) * st->M * m, cudaMemcpyDeviceToHost,
                           st->stream));
  st->d2h += (int64_t)sizeof(double) * st->M * m;
  CUDA_TRY(cudaStreamSynchronize(st->stream));
  return SPINRP_OK;
}

extern "C" int spinrp_polarization(spinrp_state *st, int site, double *out, int64_t cap, int64_t *n) {
  if (!st) return fail(SPINRP_EINVAL, "polarization: state is NULL");
  if (site < 1 || site > st->M) return fail(SPINRP_EINVAL, "polarization: site %d outside 1..%d", site, st->M);
  if (site == 1) return copy_series(st, 0, out, cap, n);
  if (!n || (cap > 0 && !out)) return fail(SPINRP_EINVAL, "polarization: bad argument");
  if (!st->ready || !st->sites)
    return fail(SPINRP_ESTATE, "polarization: site %d needs the all-site readout (spinrp_state_set_sites)", site);
  *n = st->len;
  const int64_t m = std::min(cap, st->len);
  if (m <= 0) return SPINRP_OK;
  std::vector<double> buf((size_t)st->M * m);
  CUDA_TRY(cudaMemcpyAsync(buf.data(), st->site_series, sizeof(double) * buf.size(), cudaMemcpyDeviceToHost,
                           st->stream));
  st->d2h += (int64_t)sizeof(double) * buf.size();
  CUDA_TRY(cudaStreamSynchronize(st->stream));
  for (int64_t k = 0; k < m; ++k) out[k] = buf[k * st->M + (site - 1)];
  return SPINRP_OK;
}

extern "C" int spinrp_norm_series(spinrp_state *st, double *out, int64_t cap, int64_t *n) {
  return copy_series(st, 1, out, cap, n);
}

extern "C" int spinrp_sector_norms(spinrp_state *st, double *out, int cap, int *n) {
  if (!st || !n || (cap > 0 && !out)) return fail(SPINRP_EINVAL, "sector_norms: bad argument");
  if (!st->ready) return fail(SPINRP_ESTATE, "sector_norms: state not initialized");
  const int M = st->M;
  *n = M + 1;
  if (cap <= 0) return SPINRP_OK;
  const int nblk = init_blocks(M);  // <= the state's max_blocks rows of psites
  double *part = st->psites, *dev_out = reinterpret_cast<double *>(st->stage);
  g_launches += 2;
  if (st->prec == SPINRP_C64)
    sector_kernel<float><<<nblk, 256, 0, st->stream>>>((const float2 *)st->psi, M, part, nblk);
  else
    sector_kernel<double><<<nblk, 256, 0, st->stream>>>((const double2 *)st->psi, M, part, nblk);
  CUDA_TRY(cudaGetLastError());
  sector_finalize_kernel<<<M + 1, 256, 0, st->stream>>>(part, nblk, dev_out);
  CUDA_TRY(cudaGetLastError());
  double buf[kMaxM + 1];
  CUDA_TRY(cudaMemcpyAsync(buf, dev_out, sizeof(double) * (M + 1), cudaMemcpyDeviceToHost, st->stream));
  st->d2h += (int64_t)sizeof(double) * (M + 1);
  CUDA_TRY(cudaStreamSynchronize(st->stream));
  for (int k = 0; k < std::min(cap, M + 1); ++k) out[k] = buf[k];
  return SPINRP_OK;
}

extern "C" int spinrp_profile(spinrp_state *st, int enable) {
  if (!st) return fail(SPINRP_EINVAL, "profile: state is NULL");
  if (enable) {
    cudaStreamSynchronize(st->stream);
    prof_clear(st);
  }
  st->prof = enable != 0;
  return SPINRP_OK;
}

extern "C" int spinrp_profile_read(spinrp_state *st, int kind, double *total_ms, int64_t *launches) {
  if (!st || kind < 0 || kind > 2) return fail(SPINRP_EINVAL, "profile_read: bad argument");
  CUDA_TRY(cudaStreamSynchronize(st->stream));
  const auto &v = st->ev[kind];
  double ms = 0.0;
  for (size_t k = 0; k + 1 < v.size(); k += 2) {
    float t = 0.0f;
    CUDA_TRY(cudaEventElapsedTime(&t, v[k], v[k + 1]));
    ms += t;
  }
  if (total_ms) *total_ms = ms;
  if (launches) *launches = (int64_t)(v.size() / 2);
  return SPINRP_OK;
}

extern "C" int spinrp_state_transfer_bytes(const spinrp_state *st, int64_t *h2d, int64_t *d2h) {
  if (!st) return fail(SPINRP_EINVAL, "transfer_bytes: state is NULL");
  if (h2d) *h2d = st->h2d;
  if (d2h) *d2h = st->d2h;
  return SPINRP_OK;
}

// ---------------------------------------------------------------------------
// host self-check of the register-blocked programs
// ---------------------------------------------------------------------------
#include <complex>
#include <random>

namespace {
using cplx = std::complex<double>;

void check_rotate(std::vector<cplx> &A, int u, int v, int coef) {
  const double th = 0.1 + 0.013 * coef, c = std::cos(th), s = std::sin(th);
  const size_t T = A.size();
  for (size_t t = 0; t < T; ++t) {
    if (((t >> u) & 1) != 1 || ((t >> v) & 1) != 0) continue;
    const size_t w = t ^ (size_t(1) << u) ^ (size_t(1) << v);
    const cplx a = A[t], b = A[w];
    A[t] = c * a - cplx(0, s) * b;
    A[w] = c * b - cplx(0, s) * a;
  }
}
void check_diag(std::vector<cplx> &A, int arg) {
  for (size_t t = 0; t < A.size(); ++t) {
    const double ph = 0.3 * double((t * 2654435761u) % 1000u) / 1000.0 + 0.7 * arg;
    A[t] *= cplx(std::cos(ph), std::sin(ph));
  }
}
double check_reduce(const std::vector<cplx> &A) {
  double r = 0.0;
  for (size_t t = 0; t < A.size(); ++t) r += std::norm(A[t]) * double(t % 7 + 1);
  return r;
}

// Host replay of sweep2_kernel's index arithmetic for one pass and one block:
// global addresses in range (and 16-byte aligned for the vector stores),
// shared-memory slots in range and each touched exactly once per stage.
uint32_t host_slot(uint32_t t) { return t ^ (((t >> 4) ^ (t >> 8) ^ (t >> 12)) & 15u); }

std::string audit_sweep2(const PassDesc &d, const PhaseDesc *phases, int M, uint64_t block, int rb,
                         size_t nphases_all, size_t nrops_all, bool oriented = false) {
  const int K = d.K, nt = 1 << (K - rb), lognt = K - rb;
  if (d.nphases < 0 || d.nphases > kMaxPassPhases || d.nrops < 0 || d.nrops > kMaxPassOps ||
      d.phase0 < 0 || (size_t)d.phase0 + d.nphases > nphases_all || d.rop0 < 0 ||
      (size_t)d.rop0 + d.nrops > nrops_all)
    return "program staging out of range";
  for (int p = 0; p < d.nphases; ++p) {
    const int o0 = phases[d.phase0 + p].op0 - d.rop0;
    if (o0 < 0 || o0 + phases[d.phase0 + p].nops > d.nrops) return "phase op range";
  }
  const uint32_t T = 1u << K;
  uint64_t base = 0;
  for (int k = 0; k < M - K; ++k) base |= ((block >> k) & 1ull) << d.outer_pos[k];
  auto phys = [&](uint32_t t) {
    uint64_t o = base;
    for (int q = 0; q < K; ++q) o |= (uint64_t)((t >> q) & 1u) << d.tile_pos[q];
    return o;
  };
  const uint64_t N = 1ull << M;
  char buf[160];
  if (M - K > 31) return "more than 31 outer bits";
  // the kernel's block origin: OR of lane contributions
  uint64_t kbase = 0;
  for (int lane = 0; lane < 32; ++lane)
    if (lane < M - K) kbase |= ((block >> lane) & 1ull) << d.outer_pos[lane];
  if (kbase != base) return "block origin";
  auto gray = [](int g) { return g ^ (g >> 1); };
  auto low_bit = [](int g) { int k = 0; while (!((g >> k) & 1)) ++k; return k; };
  // load: amplitude t = tid + nt*gray(g), walked as the kernel walks it
  std::vector<char> seen(T, 0);
  for (int tid = 0; tid < nt; ++tid) {
    uint64_t off = 0;
    for (int k = 0; k < lognt; ++k) if ((tid >> k) & 1) off |= 1ull << d.tile_pos[k];
    const int64_t elem0 = (int64_t)(base + off);
    const uint32_t s0 = host_slot((uint32_t)tid);
    int64_t elem = elem0;
    uint32_t s = s0;
    for (int g = 0; g < (1 << rb); ++g) {
      if ((g & 7) == 0) {  // a run of eight starts from the origin
        elem = elem0, s = s0;
        for (int k = 0; k < rb; ++k)
          if ((gray(g) >> k) & 1) elem += (int64_t)1 << d.tile_pos[lognt + k], s ^= host_slot(1u << (lognt + k));
      } else {
        const int k = low_bit(g);
        const int64_t dg = (int64_t)1 << d.tile_pos[lognt + k];
        elem += ((gray(g) >> k) & 1) ? dg : -dg;
        s ^= host_slot(1u << (lognt + k));
      }
      const uint32_t t = ((uint32_t)gray(g) << lognt) | (uint32_t)tid;
      if (t >= T || s >= T || s != host_slot(t) || seen[s]++ || elem < 0 || (uint64_t)elem >= N ||
          (uint64_t)elem != phys(t)) {
        snprintf(buf, sizeof buf, "load index out of place (t=%u)", t);
        return buf;
      }
    }
  }
  // phases: every thread's 32-amplitude subcube, slots by linearity of the swizzle
  for (int p = 0; p < d.nphases; ++p) {
    const PhaseDesc &ph = phases[d.phase0 + p];
    std::fill(seen.begin(), seen.end(), 0);
    for (int tid = 0; tid < nt; ++tid) {
      uint32_t t0 = 0;
      for (int k = 0; k < 5; ++k) t0 |= ((uint32_t)(tid >> k) & 1u) << ph.lanes[k];
      for (int k = 0; k < lognt - 5; ++k) t0 |= ((uint32_t)(tid >> (5 + k)) & 1u) << ph.warps[k];
      uint32_t s0 = 0;  // as the kernel forms it: XOR of the thread-index bits' slots
      for (int b = 0; b < lognt; ++b)
        if ((tid >> b) & 1) s0 ^= ph.tslot[b];
      for (int i = 0; i < (1 << rb); ++i) {
        uint32_t t = t0, s = s0;
        for (int k = 0; k < rb; ++k)
          if ((i >> k) & 1) t |= 1u << ph.rb[k], s ^= ph.sm[k];
        if (t >= T || s != host_slot(t) || s >= T || seen[s]++) {
          snprintf(buf, sizeof buf, "phase %d subcube index out of place (t=%u)", p, t);
          return buf;
        }
      }
      // the kernel's walk over its packs: byte offsets, runs of eight (an
      // oriented phase walks all 2^rb words over every register bit)
      const uint32_t ob = s0 << 3;
      uint32_t o = ob;
      if (oriented) {
        for (int g = 0; g < (1 << rb); ++g) {
          const int j = gray(g);
          if ((g & 7) == 0) {
            o = ob;
            for (int k = 0; k < rb; ++k)
              if ((j >> k) & 1) o ^= (uint32_t)ph.sm[k] << 3;
          } else {
            o ^= (uint32_t)ph.sm[low_bit(g)] << 3;
          }
          uint32_t s = s0;
          for (int k = 0; k < rb; ++k)
            if ((j >> k) & 1) s ^= ph.sm[k];
          if (o != (s << 3) || (o >> 3) >= T) {
            snprintf(buf, sizeof buf, "phase %d oriented walk out of place (g=%d)", p, g);
            return buf;
          }
        }
        continue;
      }
      for (int g = 0; g < (1 << (rb - 1)); ++g) {
        const int j = gray(g);
        if ((g & 7) == 0) {
          o = ob;
          for (int k = 0; k < rb - 1; ++k)
            if ((j >> k) & 1) o ^= (uint32_t)ph.sm[1 + k] << 3;
        } else {
          o ^= (uint32_t)ph.sm[1 + low_bit(g)] << 3;
        }
        uint32_t s = s0;
        for (int k = 0; k < rb - 1; ++k)
          if ((j >> k) & 1) s ^= ph.sm[1 + k];
        if (o != (s << 3) || ((o ^ ((uint32_t)ph.sm[0] << 3)) >> 3) >= T || (o >> 3) >= T) {
          snprintf(buf, sizeof buf, "phase %d pack walk out of place (g=%d)", p, g);
          return buf;
        }
      }
    }
  }
  // store: output chunk 2*(tid + nt*gray(g)) of two amplitudes, 16-byte
  // aligned, walked as the kernel walks it
  std::fill(seen.begin(), seen.end(), 0);
  for (int tid = 0; tid < nt; ++tid) {
    uint64_t off_lo = 0;
    uint32_t pin_lo = 0;
    for (int k = 0; k < lognt; ++k)
      if ((tid >> k) & 1) off_lo |= 1ull << d.tile_pos[d.store_bit[k]], pin_lo |= 1u << d.perm[d.store_bit[k]];
    const int64_t elem0 = (int64_t)(base + off_lo);
    const uint32_t so0 = host_slot(pin_lo);
    int64_t elem = elem0;
    uint32_t so = so0;
    const uint32_t sl1 = host_slot(1u << d.perm[0]);
    for (int g = 0; g < (1 << (rb - 1)); ++g) {
      if ((g & 7) == 0) {
        elem = elem0, so = so0;
        for (int k = 0; k < rb - 1; ++k)
          if ((gray(g) >> k) & 1)
            elem += (int64_t)1 << d.tile_pos[d.store_bit[lognt + k]],
                so ^= host_slot(1u << d.perm[d.store_bit[lognt + k]]);
      } else {
        const int k = low_bit(g);
        const int64_t dh = (int64_t)1 << d.tile_pos[d.store_bit[lognt + k]];
        elem += ((gray(g) >> k) & 1) ? dh : -dh;
        so ^= host_slot(1u << d.perm[d.store_bit[lognt + k]]);
      }
      // output tile index of chunk c = tid + nt * gray(g): chunk-index bit i is
      // output bit store_bit[i]; the chunk's first amplitude has output bit 0 clear
      const uint32_t c = ((uint32_t)gray(g) << lognt) | (uint32_t)tid;
      uint32_t tout = 0;
      for (int i = 0; i + 1 < K; ++i)
        if ((c >> i) & 1) tout |= 1u << d.store_bit[i];
      uint32_t tin = 0;
      for (int q = 1; q < K; ++q) tin |= ((tout >> q) & 1u) << d.perm[q];
      const uint32_t tin1 = tin | (1u << d.perm[0]);
      if (elem < 0 || (elem & 1) || (uint64_t)elem + 1 >= N || (uint64_t)elem != phys(tout) || tin >= T ||
          tin1 >= T || so != host_slot(tin) || (so ^ sl1) != host_slot(tin1) || seen[so]++ ||
          seen[so ^ sl1]++) {
        snprintf(buf, sizeof buf, "store index out of place (t=%u)", tout);
        return buf;
      }
    }
  }
  return "";
}

// Host emulation (FP64) of an oriented pass's register arithmetic, thread by
// thread and word by word as oriented_phase forms it: the stored words
// (Re, Im) or (Im, Re), the coefficient pairs (t, -t), (-s, s) negated by
// the parity of the first NB register bits of j and the thread's own
// orientation; diagonal ops conjugated for odd amplitudes.  Checked against
// the plain program's result A1 from the same start A0, for both
// orientations of the tile's outer bits.
std::string emulate_oriented(const PassDesc &d, const PhaseDesc *phases, const ROp *rops, int rb, int K,
                             const std::vector<cplx> &A0, const std::vector<cplx> &A1) {
  const int NA = 1 << rb, lognt = K - rb, nt = 1 << lognt;
  const size_t T = A0.size();
  auto par = [](uint64_t x) { return (int)(__builtin_popcountll(x) & 1); };
  for (int outer = 0; outer < 2; ++outer) {
    std::vector<double> X(T), Y(T);  // stored words
    auto ori = [&](size_t t) { return par(t & d.black_tile) ^ outer; };
    for (size_t t = 0; t < T; ++t) {
      const bool o = ori(t);
      X[t] = o ? A0[t].imag() : A0[t].real();
      Y[t] = o ? A0[t].real() : A0[t].imag();
    }
    for (int p = 0; p < d.nphases; ++p) {
      const PhaseDesc &ph = phases[d.phase0 + p];
      for (int k = 0; k < ph.nops; ++k) {
        const ROp &r = rops[ph.op0 + k];
        if (r.kind == OP_DIAG) {
          for (size_t t = 0; t < T; ++t) {
            const double phs = 0.3 * double((t * 2654435761u) % 1000u) / 1000.0 + 0.7 * r.arg;
            const double c = std::cos(phs), sn = ori(t) ? -std::sin(phs) : std::sin(phs);
            const double x = X[t], y = Y[t];
            X[t] = c * x - sn * y, Y[t] = sn * x + c * y;
          }
          continue;
        }
        if (r.kind != OP_GATE) continue;
        const int NB = ph.nb, ku = r.combo >> 3, kv = r.combo & 7;
        if (!((kOrientNbMask(rb) >> NB) & 1u) || ku >= NB || kv < NB || kv >= rb) return "combo out of range";
        for (int b = 0; b < rb; ++b)
          if ((int)((d.black_tile >> ph.rb[b]) & 1u) != (b < NB ? 1 : 0)) return "register bits out of colour order";
        const double th = 0.1 + 0.013 * r.coef, tt = std::tan(0.5 * th), ss = std::sin(th);
        for (int tid = 0; tid < nt; ++tid) {
          uint32_t t0 = 0;
          for (int b = 0; b < 5; ++b) t0 |= ((uint32_t)(tid >> b) & 1u) << ph.lanes[b];
          for (int b = 0; b < lognt - 5; ++b) t0 |= ((uint32_t)(tid >> (5 + b)) & 1u) << ph.warps[b];
          const int tp = par(t0 & d.black_tile) ^ outer;
          auto tix = [&](int j) {
            uint32_t t = t0;
            for (int b = 0; b < rb; ++b)
              if ((j >> b) & 1) t |= 1u << ph.rb[b];
            return t;
          };
          for (int j = 0; j < NA; ++j) {
            if (!((j >> ku) & 1) || ((j >> kv) & 1)) continue;
            const int sg = par((uint64_t)j & ((1u << NB) - 1u)) ^ tp;
            const double T0 = sg ? -tt : tt, T1 = -T0, S0 = sg ? ss : -ss, S1 = -S0;
            const uint32_t a = tix(j), b = tix(j ^ (1 << ku) ^ (1 << kv));
            X[a] += T0 * X[b], Y[a] += T1 * Y[b];
            X[b] += S0 * X[a], Y[b] += S1 * Y[a];
            X[a] += T0 * X[b], Y[a] += T1 * Y[b];
          }
        }
      }
    }
    double err = 0.0, ref = 0.0;
    for (size_t t = 0; t < T; ++t) {
      const bool o = ori(t);
      const cplx v(o ? Y[t] : X[t], o ? X[t] : Y[t]);
      err = std::max(err, std::abs(v - A1[t]));
      ref = std::max(ref, std::abs(A1[t]));
    }
    if (!(err <= 1e-10 * ref)) {
      char buf[96];
      snprintf(buf, sizeof buf, "packed arithmetic differs (%.3e, outer parity %d)", err, outer);
      return buf;
    }
  }
  return "";
}

// Host replay of sweep2d_kernel's (complex128) index arithmetic for one pass
// and one block, as audit_sweep2 does for the complex64 kernel: one 16-byte
// amplitude per access, 32 amplitudes per thread, slots by swizzle_slot16.
std::string audit_sweep2d(const PassDesc &d, const PhaseDesc *phases, int M, uint64_t block,
                          size_t nphases_all, size_t nrops_all) {
  constexpr int rb = 5;
  const int K = d.K, nt = 1 << (K - rb), lognt = K - rb;
  if (K < 10 || K > 13) return "tile width outside 10..13";
  if (d.nphases < 0 || d.nphases > kMaxPassPhases || d.nrops < 0 || d.nrops > kMaxPassOps ||
      d.phase0 < 0 || (size_t)d.phase0 + d.nphases > nphases_all || d.rop0 < 0 ||
      (size_t)d.rop0 + d.nrops > nrops_all)
    return "program staging out of range";
  for (int p = 0; p < d.nphases; ++p) {
    const int o0 = phases[d.phase0 + p].op0 - d.rop0;
    if (o0 < 0 || o0 + phases[d.phase0 + p].nops > d.nrops) return "phase op range";
  }
  if (M - K > 31) return "more than 31 outer bits";
  const uint32_t T = 1u << K;
  uint64_t base = 0;
  for (int k = 0; k < M - K; ++k) base |= ((block >> k) & 1ull) << d.outer_pos[k];
  auto phys = [&](uint32_t t) {
    uint64_t o = base;
    for (int q = 0; q < K; ++q) o |= (uint64_t)((t >> q) & 1u) << d.tile_pos[q];
    return o;
  };
  const uint64_t N = 1ull << M;
  char buf[160];
  auto gray = [](int g) { return g ^ (g >> 1); };
  auto low_bit = [](int g) { int k = 0; while (!((g >> k) & 1)) ++k; return k; };
  // load: amplitude t = tid + nt*gray(g), runs of eight from the origin
  std::vector<char> seen(T, 0);
  for (int tid = 0; tid < nt; ++tid) {
    uint64_t off = 0;
    for (int k = 0; k < lognt; ++k) if ((tid >> k) & 1) off |= 1ull << d.tile_pos[k];
    const int64_t elem0 = (int64_t)(base + off);
    const uint32_t s0 = swizzle_slot16((uint32_t)tid);
    int64_t elem = elem0;
    uint32_t sl = s0;
    for (int g = 0; g < (1 << rb); ++g) {
      if ((g & 7) == 0) {
        elem = elem0, sl = s0;
        for (int k = 0; k < rb; ++k)
          if ((gray(g) >> k) & 1)
            elem += (int64_t)1 << d.tile_pos[lognt + k], sl ^= swizzle_slot16(1u << (lognt + k));
      } else {
        const int k = low_bit(g);
        const int64_t dg = (int64_t)1 << d.tile_pos[lognt + k];
        elem += ((gray(g) >> k) & 1) ? dg : -dg;
        sl ^= swizzle_slot16(1u << (lognt + k));
      }
      const uint32_t t = ((uint32_t)gray(g) << lognt) | (uint32_t)tid;
      if (t >= T || sl >= T || sl != swizzle_slot16(t) || seen[sl]++ || elem < 0 || (uint64_t)elem >= N ||
          (uint64_t)elem != phys(t)) {
        snprintf(buf, sizeof buf, "load index out of place (t=%u)", t);
        return buf;
      }
    }
  }
  // phases: each thread's 32-amplitude subcube and the kernel's walk over it
  for (int p = 0; p < d.nphases; ++p) {
    const PhaseDesc &ph = phases[d.phase0 + p];
    std::fill(seen.begin(), seen.end(), 0);
    for (int tid = 0; tid < nt; ++tid) {
      uint32_t t0 = 0;
      for (int k = 0; k < 5; ++k) t0 |= ((uint32_t)(tid >> k) & 1u) << ph.lanes[k];
      for (int k = 0; k < lognt - 5; ++k) t0 |= ((uint32_t)(tid >> (5 + k)) & 1u) << ph.warps[k];
      uint32_t s0 = 0;
      for (int b = 0; b < lognt; ++b)
        if ((tid >> b) & 1) s0 ^= ph.tslot[b];
      const uint32_t ob = s0 << 4;
      uint32_t o = ob;
      for (int g = 0; g < (1 << rb); ++g) {
        const int j = gray(g);
        if ((g & 7) == 0) {
          o = ob;
          for (int k = 0; k < rb; ++k)
            if ((j >> k) & 1) o ^= (uint32_t)ph.sm[k] << 4;
        } else {
          o ^= (uint32_t)ph.sm[low_bit(g)] << 4;
        }
        uint32_t t = t0;
        for (int k = 0; k < rb; ++k)
          if ((j >> k) & 1) t |= 1u << ph.rb[k];
        if (t >= T || (o & 15u) || (o >> 4) >= T || (o >> 4) != swizzle_slot16(t) || seen[o >> 4]++) {
          snprintf(buf, sizeof buf, "phase %d subcube index out of place (t=%u)", p, t);
          return buf;
        }
      }
    }
  }
  // store: output amplitude tout = tid + nt*gray(g) takes input tile index
  // sum of bits perm[q]
  std::fill(seen.begin(), seen.end(), 0);
  for (int tid = 0; tid < nt; ++tid) {
    uint64_t off_lo = 0;
    uint32_t pin_lo = 0;
    for (int k = 0; k < lognt; ++k)
      if ((tid >> k) & 1) off_lo |= 1ull << d.tile_pos[k], pin_lo |= 1u << d.perm[k];
    const int64_t elem0 = (int64_t)(base + off_lo);
    const uint32_t so0 = swizzle_slot16(pin_lo);
    int64_t elem = elem0;
    uint32_t so = so0;
    for (int g = 0; g < (1 << rb); ++g) {
      if ((g & 7) == 0) {
        elem = elem0, so = so0;
        for (int k = 0; k < rb; ++k)
          if ((gray(g) >> k) & 1)
            elem += (int64_t)1 << d.tile_pos[lognt + k], so ^= swizzle_slot16(1u << d.perm[lognt + k]);
      } else {
        const int k = low_bit(g);
        const int64_t dh = (int64_t)1 << d.tile_pos[lognt + k];
        elem += ((gray(g) >> k) & 1) ? dh : -dh;
        so ^= swizzle_slot16(1u << d.perm[lognt + k]);
      }
      const uint32_t tout = ((uint32_t)gray(g) << lognt) | (uint32_t)tid;
      uint32_t tin = 0;
      for (int q = 0; q < K; ++q) tin |= ((tout >> q) & 1u) << d.perm[q];
      if (elem < 0 || (uint64_t)elem >= N || (uint64_t)elem != phys(tout) || tin >= T ||
          so != swizzle_slot16(tin) || seen[so]++) {
        snprintf(buf, sizeof buf, "store index out of place (t=%u)", tout);
        return buf;
      }
    }
  }
  return "";
}
}  // namespace

extern "C" int spinrp_system_orientation(const spinrp_system *sys, int prec, uint64_t *black) {
  if (!sys || !black || (prec != SPINRP_C64 && prec != SPINRP_C128))
    return fail(SPINRP_EINVAL, "system_orientation: bad argument");
  Plan plan;
  PassSet ps;
  int mb = 0;
  const int rc = plan_state(*sys, prec, &plan, &ps, &mb);
  if (rc) return rc;
  *black = ps.oriented ? ps.black : 0;
  return SPINRP_OK;
}

extern "C" int spinrp_system_plan_check(const spinrp_system *sys, int prec, double *phases_per_sweep,
                                        double *gates_per_phase) {
  if (!sys || (prec != SPINRP_C64 && prec != SPINRP_C128))
    return fail(SPINRP_EINVAL, "plan_check: bad argument");
  Plan plan;
  PassSet ps;
  int mb = 0;
  int rc = plan_state(*sys, prec, &plan, &ps, &mb);
  if (rc) return rc;
  if (phases_per_sweep) *phases_per_sweep = 0.0;
  if (gates_per_phase) *gates_per_phase = 0.0;
  const int K = plan.K;
  if (!ps.phased) return SPINRP_OK;
  const size_t T = size_t(1) << K;
  std::mt19937_64 rng(12345);
  std::normal_distribution<double> nd;
  long nphase = 0, ngate_phase = 0, ngates = 0;
  for (size_t pi = 0; pi < ps.desc.size(); ++pi) {
    const PassDesc &d = ps.desc[pi];
    const uint64_t nblocks = 1ull << (plan.M - K);
    for (uint64_t blk : {uint64_t(0), nblocks / 3, nblocks - 1}) {
      const std::string e =
          prec == SPINRP_C64
              ? audit_sweep2(d, ps.phases.data(), plan.M, blk, ps.rb, ps.phases.size(), ps.rops.size(),
                             ps.oriented)
              : audit_sweep2d(d, ps.phases.data(), plan.M, blk, ps.phases.size(), ps.rops.size());
      if (!e.empty()) return fail(SPINRP_EINVAL, "plan_check: pass %zu block %llu: %s", pi,
                                  (unsigned long long)blk, e.c_str());
    }
    std::vector<cplx> A(T), B;
    for (auto &x : A) x = cplx(nd(rng), nd(rng));
    B = A;
    const std::vector<cplx> A0 = A;
    std::vector<double> ra, rb;
    for (int k = 0; k < d.nops; ++k) {
      const Op &op = ps.ops[d.op0 + k];
      if (op.kind == OP_GATE) check_rotate(A, op.u, op.v, op.coef);
      else if (op.kind == OP_DIAG) check_diag(A, op.arg);
      else ra.push_back(check_reduce(A));
    }
    std::vector<int> KU, KV;  // combo -> register-bit pair
    if (ps.oriented) {
      for (int c = 0; c < 64; ++c) KU.push_back(c >> 3), KV.push_back(c & 7);
    } else {
      for (int a = 0; a < ps.rb; ++a)
        for (int bb = a + 1; bb < ps.rb; ++bb) KU.push_back(a), KV.push_back(bb);
    }
    for (int p = 0; p < d.nphases; ++p) {
      const PhaseDesc &ph = ps.phases[d.phase0 + p];
      uint32_t seen = 0;
      for (int k = 0; k < ps.rb; ++k) seen |= 1u << ph.rb[k];
      for (int k = 0; k < 5; ++k) seen |= 1u << ph.lanes[k];
      for (int k = 0; k < K - ps.rb - 5; ++k) seen |= 1u << ph.warps[k];
      if (seen != (1u << K) - 1u || __builtin_popcount(seen) != K)
        return fail(SPINRP_EINVAL, "plan_check: pass %zu phase %d does not partition the tile bits", pi, p);
      int g = 0;
      for (int k = 0; k < ph.nops; ++k) {
        const ROp &r = ps.rops[ph.op0 + k];
        if (r.kind == OP_GATE) {
          check_rotate(B, ph.rb[KU[r.combo]], ph.rb[KV[r.combo]], r.coef);
          ++g;
        } else if (r.kind == OP_DIAG) {
          if (ph.nops != 1) return fail(SPINRP_EINVAL, "plan_check: diagonal op shares a phase");
          check_diag(B, r.arg);
        } else {
          rb.push_back(check_reduce(B));
        }
      }
      ++nphase;
      if (g) ++ngate_phase, ngates += g;
    }
    double err = 0.0, ref = 0.0;
    for (size_t t = 0; t < T; ++t) err = std::max(err, std::abs(A[t] - B[t])), ref = std::max(ref, std::abs(A[t]));
    if (!(err <= 1e-10 * ref)) return fail(SPINRP_EINVAL, "plan_check: pass %zu differs (%.3e)", pi, err);
    if (ps.oriented) {
      const std::string e = emulate_oriented(d, ps.phases.data(), ps.rops.data(), ps.rb, K, A0, A);
      if (!e.empty()) return fail(SPINRP_EINVAL, "plan_check: pass %zu oriented: %s", pi, e.c_str());
    }
    if (ra.size() != rb.size()) return fail(SPINRP_EINVAL, "plan_check: pass %zu reductions differ", pi);
    for (size_t k = 0; k < ra.size(); ++k)
      if (std::abs(ra[k] - rb[k]) > 1e-9 * std::abs(ra[k]))
        return fail(SPINRP_EINVAL, "plan_check: pass %zu reduction %zu at a different point", pi, k);
  }
  if (phases_per_sweep) *phases_per_sweep = ps.desc.empty() ? 0.0 : double(nphase) / ps.desc.size();
  if (gates_per_phase) *gates_per_phase = ngate_phase ? double(ngates) / ngate_phase : 0.0;
  return SPINRP_OK;
}

// ---------------------------------------------------------------------------
// batches
// ---------------------------------------------------------------------------
namespace {

// Mean and standard deviation over jobs of P(t_k) (FP64, two passes).
__global__ void ensemble_kernel(const JobPtrs *__restrict__ jobs, int njobs, int64_t len,
                                double *__restrict__ out) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < len;
       t += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < njobs; ++j) s += jobs[j].series[2 * t];
    const double mean = s / njobs;
    double v = 0.0;
    for (int j = 0; j < njobs; ++j) {
      const double d = jobs[j].series[2 * t] - mean;
      v += d * d;
    }
    out[t] = mean;
    out[len + t] = sqrt(v / njobs);
  }
}

struct BatchGroup {
  std::vector<int> jobs;  // batch job indices
  int M = 0, nb = 0, max_blocks = 0;
  unsigned pipe_blocks = 0;  // blocks of the pipelined sweep for this group, 0 when it does not apply
  bool has_diag = false;
  Plan plan;
  PassSet ps;
  LaunchCtx ctx;
  std::vector<uint8_t> logical_of;
  unsigned char *dev = nullptr;
  JobPtrs *d_jobs = nullptr;
  uint64_t *d_seeds = nullptr;
};

}  // namespace

struct spinrp_batch {
  int prec = 0;
  cudaStream_t stream = nullptr;
  int64_t cap = 0, len = 0;
  bool ready = false;
  double coef_dt = NAN;
  std::vector<BatchGroup> groups;
  std::vector<JobPtrs> hjobs;  // every job's device pointers (host copy)
  JobPtrs *d_all = nullptr;    // the same table on the device (ensemble)
  double *d_ens = nullptr;     // 2 * cap doubles
  unsigned char *dev_common = nullptr;
  size_t bytes = 0;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graphs[2] = {nullptr, nullptr};
  // one persistent launch for the multi-tile groups (persist.cuh)
  bool persist = false;
  int persist_K = 0;                   // common tile width of the eligible groups (0: none)
  unsigned char *d_persist = nullptr;  // PersistPlan, queue, error word, per-job counters
  PersistPlan *h_plan = nullptr;       // host copy of the uploaded plan
  int64_t plan_steps = -1;             // steps the uploaded plan and its graph are for
  cudaGraphExec_t pgraph = nullptr;
  unsigned persist_blocks = 0;
  // pipelined sweeps of the eligible multi-tile groups (pipe_kernel)
  bool pipe_req = true;
  int *d_pipe_err = nullptr;  // their error word (in dev_common)
};

static void free_batch(spinrp_batch *b) {
  if (!b) return;
  if (b->pgraph) cudaGraphExecDestroy(b->pgraph);
  if (b->d_persist) cudaFree(b->d_persist);
  delete b->h_plan;
  for (cudaGraphExec_t g : b->graphs)
    if (g) cudaGraphExecDestroy(g);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  for (auto &g : b->groups)
    if (g.dev) cudaFree(g.dev);
  if (b->dev_common) cudaFree(b->dev_common);
  delete b;
}

// A multi-tile group can join the persistent launch: complex64 register
// programs of six register bits on 13- or 14-spin tiles (the launch's block
// size), plain storage, at most 31 outer bits, a step's sweeps in the plan's
// steady list.
static bool persist_eligible(const BatchGroup &g, int prec) {
  return prec == SPINRP_C64 && !g.ctx.resident && g.ps.phased && !g.ps.oriented && g.ps.rb == 6 &&
         (g.plan.K == 13 || g.plan.K == 14) && g.plan.M - g.plan.K <= 31 && g.plan.segments() >= 2 &&
         g.plan.sweeps_per_step() - 1 <= kMaxSteadyPasses && g.ps.head >= 0 && g.ps.join >= 0 &&
         g.ps.tail >= 0 && g.ps.mid >= 0;
}

static bool in_persist(const spinrp_batch *b, const BatchGroup &g) {
  return b->persist && b->persist_K > 0 && persist_eligible(g, b->prec) && g.plan.K == b->persist_K;
}

// The host plan of a persistent launch of `steps` Trotter steps over the
// batch's groups in the launch; false if the counts do not fit.
static bool build_persist_plan(const spinrp_batch *b, int64_t steps, PersistPlan *pp) {
  memset(pp, 0, sizeof *pp);
  std::vector<const BatchGroup *> gs;
  for (const BatchGroup &g : b->groups)
    if (in_persist(b, g)) gs.push_back(&g);
  if (gs.empty() || gs.size() > (size_t)kMaxPersistGroups) return false;
  std::stable_sort(gs.begin(), gs.end(), [](const BatchGroup *x, const BatchGroup *y) {
    return x->plan.sweeps_per_step() > y->plan.sweeps_per_step();
  });
  pp->ngroups = (int)gs.size();
  pp->steps = steps;
  int done0 = 0;
  unsigned long long cum = 0;
  for (int i = 0; i < pp->ngroups; ++i) {
    const BatchGroup &g = *gs[i];
    PersistGroup &G = pp->g[i];
    G.M = g.M;
    G.K = g.plan.K;
    G.njobs = (int)g.jobs.size();
    G.done0 = done0;
    done0 += G.njobs;
    G.S = g.plan.sweeps_per_step();
    const int64_t nsw = 1 + (int64_t)G.S * steps;
    G.tiles = 1u << (g.M - g.plan.K);
    if (nsw > (int64_t)1 << 30 || (uint64_t)nsw * G.tiles >= (uint64_t)1 << 32) return false;
    if ((uint64_t)G.njobs * G.tiles >= (uint64_t)1 << 31) return false;
    G.nsweeps = (int)nsw;
    G.head = g.ps.head;
    G.join = g.ps.join;
    G.tail = g.ps.tail;
    int q = 0;
    for (int id : g.ps.body) G.steady[q++] = id;
    G.steady[q++] = g.ps.mid;
    for (int id : g.ps.bodyr) G.steady[q++] = id;
    if (q != G.S - 1) return false;
    G.cum = cum;
    cum += (unsigned long long)G.njobs * G.tiles;
    G.passes = g.ctx.passes;
    G.phases = g.ctx.phases;
    G.jobs = g.ctx.jobs;
  }
  // regions of sweep indices with a fixed set of active groups (groups sorted
  // by sweeps per step, so by sweep count, most first)
  int nreg = 0;
  unsigned long long item = 0;
  int from = 0;
  for (int a = pp->ngroups; a >= 1; --a) {
    const int to = pp->g[a - 1].nsweeps;  // groups 0..a-1 are active below `to`
    if (to <= from) continue;
    pp->start[nreg] = from;
    pp->active[nreg] = a;
    pp->base[nreg] = item;
    pp->per[nreg] = pp->g[a - 1].cum + (unsigned long long)pp->g[a - 1].njobs * pp->g[a - 1].tiles;
    if (pp->per[nreg] >= (1ull << 32)) return false;  // items per sweep index fit 32 bits
    item += pp->per[nreg] * (unsigned long long)(to - from);
    from = to;
    ++nreg;
  }
  pp->start[nreg] = from;
  pp->nregions = nreg;
  pp->total = item;
  return nreg > 0;
}

extern "C" int spinrp_batch_create(int njobs, const spinrp_system *const *systems,
                                   const uint64_t *seeds, int prec, int64_t series_cap, void *stream,
                                   spinrp_batch **out) {
  if (!out) return fail(SPINRP_EINVAL, "batch_create: out is NULL");
  *out = nullptr;
  if (njobs < 1 || njobs > 65535 || !systems || !seeds || series_cap < 1 ||
      (prec != SPINRP_C64 && prec != SPINRP_C128))
    return fail(SPINRP_EINVAL, "batch_create: bad argument");
  spinrp_batch *b = new (std::nothrow) spinrp_batch;
  if (!b) return fail(SPINRP_ENOMEM, "batch_create: out of host memory");
  b->prec = prec;
  b->stream = (cudaStream_t)stream;
  b->cap = series_cap;
  b->hjobs.resize(njobs);
  // group jobs by sweep plan: same M, bond list, diagonal part and tile width
  for (int k = 0; k < njobs; ++k) {
    const spinrp_system *s = systems[k];
    if (!s) {
      free_batch(b);
      return fail(SPINRP_EINVAL, "batch_create: system %d is NULL", k);
    }
    int gi = -1;
    for (size_t g = 0; g < b->groups.size() && gi < 0; ++g) {
      const spinrp_system *r = systems[b->groups[g].jobs[0]];
      if (r->M == s->M && r->bonds == s->bonds && any_diag(*r) == any_diag(*s) &&
          r->tileK[prec] == s->tileK[prec])
        gi = (int)g;
    }
    if (gi < 0) {
      b->groups.emplace_back();
      gi = (int)b->groups.size() - 1;
    }
    b->groups[gi].jobs.push_back(k);
  }
  const size_t amp = prec == SPINRP_C64 ? 8 : 16;
  for (BatchGroup &g : b->groups) {
    const spinrp_system &s0 = *systems[g.jobs[0]];
    g.M = s0.M;
    g.nb = (int)s0.bonds.size();
    g.has_diag = any_diag(s0);
    int rc = plan_state(s0, prec, &g.plan, &g.ps, &g.max_blocks, (int)g.jobs.size());
    if (rc) {
      free_batch(b);
      return rc;
    }
    g.logical_of.assign(g.M, 0);
    for (int q = 0; q < g.M; ++q) g.logical_of[g.plan.pos[q]] = (uint8_t)q;
    const int n = (int)g.jobs.size(), M = g.M, nb = std::max(g.nb, 1);
    // one allocation: shared program, job table, seeds, then per-job blocks
    size_t o = 0;
    const size_t o_pass = o; o = align256(o + sizeof(PassDesc) * g.ps.desc.size());
    const size_t o_ops = o; o = align256(o + sizeof(Op) * std::max<size_t>(g.ps.ops.size(), 1));
    const size_t o_ph = o; o = align256(o + sizeof(PhaseDesc) * std::max<size_t>(g.ps.phases.size(), 1));
    const size_t o_rop = o; o = align256(o + sizeof(ROp) * std::max<size_t>(g.ps.rops.size(), 1));
    const size_t o_jobs = o; o = align256(o + sizeof(JobPtrs) * n);
    const size_t o_seeds = o; o = align256(o + sizeof(uint64_t) * n);
    const size_t o_job0 = o;
    size_t per = 0;
    const size_t p_psi = per; per = align256(per + (amp << M));
    const size_t p_series = per; per = align256(per + sizeof(double) * 2 * series_cap);
    const size_t p_part = per; per = align256(per + sizeof(double2) * g.max_blocks);
    const size_t p_tick = per; per = align256(per + 256);
    const size_t p_coef = per; per = align256(per + sizeof(GateCoef) * 2 * nb);
    const size_t p_bv = per; per = align256(per + sizeof(double) * nb);
    const size_t p_a = per; per = align256(per + sizeof(double) * M * M);
    const size_t p_q = per; per = align256(per + sizeof(uint64_t) * 2 * M * M);
    const size_t p_sops = per; per = align256(per + sizeof(ROpRes) * std::max<size_t>(g.ps.rops.size(), 1));
    const size_t total = o_job0 + per * n;
    cudaError_t e = cudaMalloc((void **)&g.dev, total);
    if (e != cudaSuccess) {
      cudaGetLastError();
      free_batch(b);
      return fail(SPINRP_ENOMEM, "batch_create: cudaMalloc(%zu): %s", total, cudaGetErrorString(e));
    }
    b->bytes += total;
    unsigned char *d = g.dev;
    g.d_jobs = (JobPtrs *)(d + o_jobs);
    g.d_seeds = (uint64_t *)(d + o_seeds);
    std::vector<JobPtrs> hj(n);
    std::vector<uint64_t> hs(n);
    std::vector<double> bv(nb), am(M * M);
    auto up = [&](void *dst, const void *src, size_t bytes) {
      return bytes ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, b->stream) : cudaSuccess;
    };
    for (int k = 0; k < n && e == cudaSuccess; ++k) {
      const spinrp_system &s = *systems[g.jobs[k]];
      unsigned char *j = d + o_job0 + per * k;
      JobPtrs &p = hj[k];
      p.psi = j + p_psi;
      p.series = (double *)(j + p_series);
      p.partials = (double2 *)(j + p_part);
      p.ticket = (unsigned *)(j + p_tick);
      p.step = (int64_t *)(j + p_tick + 64);
      p.coefs = (GateCoef *)(j + p_coef);
      p.bvals = (double *)(j + p_bv);
      p.a = (double *)(j + p_a);
      p.qdiag = (uint64_t *)(j + p_q);
      p.sops = (ROpRes *)(j + p_sops);
      hs[k] = seeds[g.jobs[k]];
      for (int q = 0; q < g.nb; ++q) bv[q] = s.b[s.bonds[q].first * M + s.bonds[q].second];
      for (int q = 0; q < M * M; ++q) am[q] = s.a[q];
      if ((e = cudaMemsetAsync(j + p_tick, 0, 256, b->stream)) == cudaSuccess &&
          (e = up(j + p_bv, bv.data(), sizeof(double) * g.nb)) == cudaSuccess)
        e = up(j + p_a, am.data(), sizeof(double) * M * M);
      if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);  // bv/am are reused
      b->hjobs[g.jobs[k]] = p;
    }
    if (e == cudaSuccess && (e = up(d + o_pass, g.ps.desc.data(), sizeof(PassDesc) * g.ps.desc.size())) == cudaSuccess &&
        (e = up(d + o_ops, g.ps.ops.data(), sizeof(Op) * g.ps.ops.size())) == cudaSuccess &&
        (e = up(d + o_ph, g.ps.phases.data(), sizeof(PhaseDesc) * g.ps.phases.size())) == cudaSuccess &&
        (e = up(d + o_rop, g.ps.rops.data(), sizeof(ROp) * g.ps.rops.size())) == cudaSuccess &&
        (e = up(g.d_jobs, hj.data(), sizeof(JobPtrs) * n)) == cudaSuccess)
      e = up(g.d_seeds, hs.data(), sizeof(uint64_t) * n);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
      free_batch(b);
      return fail(SPINRP_ECUDA, "batch_create: upload: %s", cudaGetErrorString(e));
    }
    LaunchCtx &c = g.ctx;
    c.M = M;
    c.K = g.plan.K;
    c.v2 = g.ps.phased;
    c.rb = g.ps.rb;
    c.segments = g.plan.segments();
    c.sweeps_per_step = g.plan.sweeps_per_step();
    c.ps = &g.ps;
    c.passes = (const PassDesc *)(d + o_pass);
    c.ops = (const Op *)(d + o_ops);
    c.phases = (const PhaseDesc *)(d + o_ph);
    c.rops = (const ROp *)(d + o_rop);
    c.jobs = g.d_jobs;
    if (n == 1) c.job0 = hj[0];
    c.njobs = n;
    // job k's buffers start per x k bytes after job 0's (the pipelined sweep
    // computes its addresses from that)
    c.batch0 = hj[0];
    c.job_stride = (long long)per;
    c.oriented = g.ps.oriented;
    c.resident_smem = resident_bytes(g.plan, g.ps, prec, false);
    c.resident = c.resident_smem > 0;

  }
  // the LaunchCtx keep pointers to their group's PassSet: fix them now that
  // the group vector no longer moves
  for (BatchGroup &g : b->groups) g.ctx.ps = &g.ps;
  const size_t o_perr = align256(align256(sizeof(JobPtrs) * njobs) + sizeof(double) * 2 * series_cap);
  const size_t common = o_perr + 256;
  cudaError_t e = cudaMalloc((void **)&b->dev_common, common);
  if (e == cudaSuccess) {
    b->d_all = (JobPtrs *)b->dev_common;
    b->d_ens = (double *)(b->dev_common + align256(sizeof(JobPtrs) * njobs));
    b->d_pipe_err = (int *)(b->dev_common + o_perr);
    e = cudaMemsetAsync(b->d_pipe_err, 0, 256, b->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(b->d_all, b->hjobs.data(), sizeof(JobPtrs) * njobs, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    free_batch(b);
    return fail(SPINRP_ENOMEM, "batch_create: %s", cudaGetErrorString(e));
  }
  b->bytes += common;
  int rc = prec == SPINRP_C64 ? set_smem_limits<float>() : set_smem_limits<double>();
  if (rc) {
    free_batch(b);
    return rc;
  }
  for (BatchGroup &g : b->groups) {
    if (g.ps.phased) g.ctx.prefetch_ahead = sweep2_resident(prec, g.ps.rb, g.plan.K, g.ps.oriented);
    g.pipe_blocks = g.ctx.resident ? 0 : pipe_grid(prec, g.plan, g.ps, g.M, (int)g.jobs.size());
    g.ctx.pipe_blocks = b->pipe_req ? g.pipe_blocks : 0;
    g.ctx.pipe_err = b->d_pipe_err;
  }
  // the persistent launch takes the eligible groups of the most common
  // eligible tile width (jobs counted)
  {
    int n13 = 0, n14 = 0;
    for (const BatchGroup &g : b->groups)
      if (persist_eligible(g, prec)) (g.plan.K == 13 ? n13 : n14) += (int)g.jobs.size();
    b->persist_K = n13 + n14 == 0 ? 0 : (n13 >= n14 ? 13 : 14);
  }
  if (b->persist_K) {
    const size_t bytes = align256(sizeof(PersistPlan)) + 256 + sizeof(unsigned) * (size_t)njobs;
    cudaError_t e2 = cudaMalloc((void **)&b->d_persist, bytes);
    b->h_plan = new (std::nothrow) PersistPlan;
    int per = 0, dev = 0, sms = 0;
    const int smem = 8 << b->persist_K;
    if (e2 == cudaSuccess)
      e2 = cudaFuncSetAttribute(persist_kernel<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e2 == cudaSuccess) e2 = cudaGetDevice(&dev);
    if (e2 == cudaSuccess) e2 = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e2 == cudaSuccess)
      e2 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, persist_kernel<6>, 1 << (b->persist_K - 6), smem);
    if (e2 != cudaSuccess || !b->h_plan || per < 1) {
      cudaGetLastError();
      free_batch(b);
      return fail(SPINRP_ENOMEM, "batch_create: persistent launch setup failed");
    }
    b->persist_blocks = (unsigned)(per * sms);
    b->bytes += bytes;
  }
  *out = b;
  return SPINRP_OK;
}

extern "C" void spinrp_batch_destroy(spinrp_batch *b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  free_batch(b);
}

extern "C" int spinrp_batch_info(const spinrp_batch *b, size_t *device_bytes, int *groups) {
  if (!b) return fail(SPINRP_EINVAL, "batch_info: batch is NULL");
  if (device_bytes) *device_bytes = b->bytes;
  if (groups) *groups = (int)b->groups.size();
  return SPINRP_OK;
}

static LayoutArg group_layout(const BatchGroup &g) {
  LayoutArg la;
  memset(&la, 0, sizeof la);
  for (int p = 0; p < g.M; ++p) la.logical_of[p] = g.logical_of[p];
  return la;
}

static int batch_init(spinrp_batch *b, int kind) {
  if (!b) return fail(SPINRP_EINVAL, "batch_init: batch is NULL");
  for (BatchGroup &g : b->groups) {
    const dim3 grid(init_blocks(g.M), (unsigned)g.jobs.size());
    ++g_launches;
    if (b->prec == SPINRP_C64)
      init_kernel<float><<<grid, 256, 0, b->stream>>>(g.d_jobs, g.M, group_layout(g), 0, g.d_seeds, kind,
                                                      g.ps.oriented ? g.ps.black : 0ull);
    else
      init_kernel<double><<<grid, 256, 0, b->stream>>>(g.d_jobs, g.M, group_layout(g), 0, g.d_seeds, kind, 0);
    CUDA_TRY(cudaGetLastError());
  }
  b->len = 1;
  b->ready = true;
  return SPINRP_OK;
}

extern "C" int spinrp_batch_init_random_phase(spinrp_batch *b) { return batch_init(b, INIT_ENTANGLED); }

extern "C" int spinrp_batch_init_product_phase(spinrp_batch *b) { return batch_init(b, INIT_PRODUCT); }

// Device layout of b->d_persist: the plan, then (at +align256(plan)) the
// queue counter (8 bytes), the error word (at +64) and the per-job counters
// (at +256).
static unsigned long long *persist_queue(spinrp_batch *b) {
  return (unsigned long long *)(b->d_persist + align256(sizeof(PersistPlan)));
}
static int *persist_err(spinrp_batch *b) { return (int *)((unsigned char *)persist_queue(b) + 64); }
static unsigned *persist_done(spinrp_batch *b) { return (unsigned *)((unsigned char *)persist_queue(b) + 256); }

// The multi-tile groups' `steps` Trotter steps as one persistent launch,
// replayed from a CUDA graph (counters cleared, then the launch) captured for
// this step count.
static int persist_evolve(spinrp_batch *b, int64_t steps) {
  int njobs = 0;
  for (const BatchGroup &g : b->groups)
    if (in_persist(b, g)) njobs += (int)g.jobs.size();
  if (b->plan_steps != steps) {
    if (!build_persist_plan(b, steps, b->h_plan))
      return fail(SPINRP_EUNSUPPORTED, "batch_evolve: persistent plan does not fit (%lld steps)", (long long)steps);
    CUDA_TRY(cudaMemcpyAsync(b->d_persist, b->h_plan, sizeof(PersistPlan), cudaMemcpyHostToDevice, b->stream));
    CUDA_TRY(cudaStreamSynchronize(b->stream));
    if (b->pgraph) cudaGraphExecDestroy(b->pgraph), b->pgraph = nullptr;
    b->plan_steps = steps;
  }
  if (!b->pgraph) {
    if (!b->cap_stream) CUDA_TRY(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
    CUDA_TRY(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaMemsetAsync(persist_queue(b), 0, 256 + sizeof(unsigned) * (size_t)njobs, b->cap_stream);
    const unsigned nt = 1u << (b->persist_K - 6);
    persist_kernel<6><<<b->persist_blocks, nt, size_t(8) << b->persist_K, b->cap_stream>>>(
        (const PersistPlan *)b->d_persist, persist_queue(b), persist_done(b), persist_err(b), b->persist_blocks);
    cudaGraph_t gr = nullptr;
    const cudaError_t e = cudaStreamEndCapture(b->cap_stream, &gr);
    if (e != cudaSuccess) {
      if (gr) cudaGraphDestroy(gr);
      cudaGetLastError();
      return fail(SPINRP_ECUDA, "batch_evolve: persistent graph capture: %s", cudaGetErrorString(e));
    }
    const cudaError_t e2 = cudaGraphInstantiate(&b->pgraph, gr, 0);
    cudaGraphDestroy(gr);
    if (e2 != cudaSuccess) {
      b->pgraph = nullptr;
      return fail(SPINRP_ECUDA, "batch_evolve: persistent graph instantiate: %s", cudaGetErrorString(e2));
    }
  }
  CUDA_TRY(cudaGraphLaunch(b->pgraph, b->stream));
  ++g_launches;
  return SPINRP_OK;
}

// SPINRP_ETIMEOUT when a wait of the last persistent launch gave up
// (synchronizes the batch's stream).
static int persist_check(spinrp_batch *b) {
  int err = 0, perr = 0;
  const bool persisted = b->d_persist && b->plan_steps >= 0;
  if (persisted) CUDA_TRY(cudaMemcpyAsync(&err, persist_err(b), sizeof err, cudaMemcpyDeviceToHost, b->stream));
  if (b->d_pipe_err) CUDA_TRY(cudaMemcpyAsync(&perr, b->d_pipe_err, sizeof perr, cudaMemcpyDeviceToHost, b->stream));
  CUDA_TRY(cudaStreamSynchronize(b->stream));
  if (err) return fail(SPINRP_ETIMEOUT, "batch: a persistent-launch wait timed out; the series are invalid");
  if (perr) return fail(SPINRP_ETIMEOUT, "batch: a wait of a pipelined sweep gave up; the series are invalid");
  return SPINRP_OK;
}

extern "C" int spinrp_batch_persist_timeout_check(spinrp_batch *b, int64_t steps, double *seconds) {
  if (!b || steps < 1) return fail(SPINRP_EINVAL, "batch_persist_timeout_check: bad argument");
  if (!b->persist_K || !b->ready) return fail(SPINRP_ESTATE, "batch_persist_timeout_check: no persistent groups");
  PersistPlan pp;
  if (!build_persist_plan(b, steps, &pp) || pp.nregions < 1 || pp.start[1] < 2)
    return fail(SPINRP_EUNSUPPORTED, "batch_persist_timeout_check: plan too small");
  // the plan on the device; the queue starts at the first item of sweep 1,
  // so the sweep-0 tiles every item waits for never run
  CUDA_TRY(cudaMemcpyAsync(b->d_persist, &pp, sizeof pp, cudaMemcpyHostToDevice, b->stream));
  b->plan_steps = -1;  // the next evolve uploads its own plan and graph
  if (b->pgraph) cudaGraphExecDestroy(b->pgraph), b->pgraph = nullptr;
  int njobs = 0;
  for (const BatchGroup &g : b->groups)
    if (in_persist(b, g)) njobs += (int)g.jobs.size();
  CUDA_TRY(cudaMemsetAsync(persist_queue(b), 0, 256 + sizeof(unsigned) * (size_t)njobs, b->stream));
  const unsigned long long first = pp.per[0];
  CUDA_TRY(cudaMemcpyAsync(persist_queue(b), &first, sizeof first, cudaMemcpyHostToDevice, b->stream));
  cudaEvent_t e0, e1;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  cudaEventRecord(e0, b->stream);
  const unsigned nt = 1u << (b->persist_K - 6);
  persist_kernel<6><<<b->persist_blocks, nt, size_t(8) << b->persist_K, b->stream>>>(
      (const PersistPlan *)b->d_persist, persist_queue(b), persist_done(b), persist_err(b), b->persist_blocks);
  cudaEventRecord(e1, b->stream);
  ++g_launches;
  const cudaError_t le = cudaGetLastError();
  int err = 0;
  cudaError_t ce = cudaMemcpyAsync(&err, persist_err(b), sizeof err, cudaMemcpyDeviceToHost, b->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(b->stream);
  float ms = 0.f;
  if (ce == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (le != cudaSuccess || ce != cudaSuccess)
    return fail(SPINRP_ECUDA, "batch_persist_timeout_check: %s", cudaGetErrorString(le != cudaSuccess ? le : ce));
  if (seconds) *seconds = ms / 1e3;
  // clear the error word again: the batch's series are unchanged (no tile ran)
  CUDA_TRY(cudaMemsetAsync(persist_err(b), 0, sizeof(int), b->stream));
  CUDA_TRY(cudaStreamSynchronize(b->stream));
  return err ? fail(SPINRP_ETIMEOUT, "batch_persist_timeout_check: the waits ran out as intended")
             : fail(SPINRP_ECUDA, "batch_persist_timeout_check: no wait ran out");
}

extern "C" int spinrp_batch_set_pipeline(spinrp_batch *b, int on) {
  if (!b || (on != 0 && on != 1)) return fail(SPINRP_EINVAL, "batch_set_pipeline: bad argument");
  if (b->pipe_req != (on != 0)) {
    // cached graphs hold the launches of the other sweep kernel
    for (cudaGraphExec_t &g : b->graphs)
      if (g) cudaGraphExecDestroy(g), g = nullptr;
    b->pipe_req = on != 0;
    for (BatchGroup &g : b->groups) g.ctx.pipe_blocks = b->pipe_req ? g.pipe_blocks : 0;
  }
  return SPINRP_OK;
}

extern "C" int spinrp_batch_pipeline(const spinrp_batch *b, int *groups) {
  if (!b || !groups) return fail(SPINRP_EINVAL, "batch_pipeline: bad argument");
  int n = 0;
  for (const BatchGroup &g : b->groups)
    if (b->pipe_req && g.pipe_blocks && !(b->persist && in_persist(b, g))) ++n;
  *groups = n;
  return SPINRP_OK;
}

extern "C" int spinrp_batch_set_persistent(spinrp_batch *b, int on) {
  if (!b || (on != 0 && on != 1)) return fail(SPINRP_EINVAL, "batch_set_persistent: bad argument");
  b->persist = on != 0;
  return SPINRP_OK;
}

extern "C" int spinrp_batch_evolve(spinrp_batch *b, double dt, int64_t steps, int order) {
  if (!b) return fail(SPINRP_EINVAL, "batch_evolve: batch is NULL");
  if (order != 2) return fail(SPINRP_EUNSUPPORTED, "batch_evolve: only order 2 is implemented");
  if (!b->ready) return fail(SPINRP_ESTATE, "batch_evolve: batch not initialized");
  if (!std::isfinite(dt) || steps < 0) return fail(SPINRP_EINVAL, "batch_evolve: bad dt or steps");
  if (steps == 0) return SPINRP_OK;
  if (b->len + steps > b->cap)
    return fail(SPINRP_EINVAL, "batch_evolve: series capacity %lld exceeded", (long long)b->cap);
  if (!(dt == b->coef_dt)) {
    for (BatchGroup &g : b->groups) {
      const unsigned n = (unsigned)g.jobs.size();
      if (g.nb > 0) {
        ++g_launches;
        coef_kernel<<<dim3((2 * g.nb + 127) / 128, n), 128, 0, b->stream>>>(g.d_jobs, g.nb, dt);
        CUDA_TRY(cudaGetLastError());
      }
      if (g.ps.phased && b->prec == SPINRP_C64 && !g.ps.rops.empty()) {
        const int nr = (int)g.ps.rops.size();
        ++g_launches;
        resolve_ops_kernel<<<dim3((nr + 127) / 128, n), 128, 0, b->stream>>>(g.d_jobs, g.ctx.rops, nr);
        CUDA_TRY(cudaGetLastError());
      }
      if (g.has_diag) {
        ++g_launches;
        diag_kernel<<<dim3((2 * g.M * g.M + 127) / 128, n), 128, 0, b->stream>>>(g.d_jobs, group_layout(g),
                                                                                  g.M, dt);
        CUDA_TRY(cudaGetLastError());
      }
    }
    b->coef_dt = dt;
  }
  std::vector<LaunchCtx> cs;
  bool any_persist = false;
  for (BatchGroup &g : b->groups) {
    if (in_persist(b, g)) any_persist = true;
    else cs.push_back(g.ctx);
  }
  if (!cs.empty()) {
    const int rc = b->prec == SPINRP_C64
                       ? run_steps<float>(cs, b->stream, steps, true, &b->cap_stream, b->graphs)
                       : run_steps<double>(cs, b->stream, steps, true, &b->cap_stream, b->graphs);
    if (rc) return rc;
  }
  if (any_persist) {
    const int rc = persist_evolve(b, steps);
    if (rc) return rc;
  }
  b->len += steps;
  return SPINRP_OK;
}

extern "C" int spinrp_batch_polarization(spinrp_batch *b, int job, double *out, int64_t cap, int64_t *n) {
  if (!b || !n || job < 0 || job >= (int)b->hjobs.size() || (cap > 0 && !out))
    return fail(SPINRP_EINVAL, "batch_polarization: bad argument");
  *n = b->len;
  const int64_t m = std::min(cap, b->len);
  if (m <= 0) return SPINRP_OK;
  if (int rc = persist_check(b)) return rc;
  std::vector<double> buf(2 * m);
  CUDA_TRY(cudaMemcpyAsync(buf.data(), b->hjobs[job].series, sizeof(double) * 2 * m,
                           cudaMemcpyDeviceToHost, b->stream));
  CUDA_TRY(cudaStreamSynchronize(b->stream));
  for (int64_t k = 0; k < m; ++k) out[k] = buf[2 * k];
  return SPINRP_OK;
}

extern "C" int spinrp_batch_ensemble(spinrp_batch *b, double *mean, double *stddev, int64_t cap,
                                     int64_t *n) {
  if (!b || !n) return fail(SPINRP_EINVAL, "batch_ensemble: bad argument");
  *n = b->len;
  const int64_t len = b->len, m = std::min(cap, len);
  if (len <= 0 || m <= 0) return SPINRP_OK;
  if (int rc = persist_check(b)) return rc;
  ++g_launches;
  ensemble_kernel<<<(unsigned)((len + 127) / 128), 128, 0, b->stream>>>(b->d_all, (int)b->hjobs.size(),
                                                                          len, b->d_ens);
  CUDA_TRY(cudaGetLastError());
  std::vector<double> buf(2 * len);
  CUDA_TRY(cudaMemcpyAsync(buf.data(), b->d_ens, sizeof(double) * 2 * len, cudaMemcpyDeviceToHost, b->stream));
  CUDA_TRY(cudaStreamSynchronize(b->stream));
  for (int64_t k = 0; k < m; ++k) {
    if (mean) mean[k] = buf[k];
    if (stddev) stddev[k] = buf[len + k];
  }
  return SPINRP_OK;
}
