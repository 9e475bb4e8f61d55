// planner.cpp -- cuts the forward half step of the Trotter product into
// shared-memory tile sweeps.
//
// The forward half step applies the flip-flop bonds in canonical order
// g_0, g_1, ..., g_{B-1}.  Two gates on disjoint spin pairs commute exactly, so
// any order that keeps, for every spin, the sequence of gates touching it is
// the same operator.  The planner exploits this freedom (and nothing else): it
// greedily grows a set Q of K spins and takes every gate that becomes
// applicable using spins of Q only; that set of gates is one segment (one
// device sweep over 2^(M-K) tiles of 2^K amplitudes).  It repeats until every
// gate is placed.  The reverse half step reuses the segments backwards.
//
// Coalescing: every tile must contain the c lowest physical bits, so that a
// tile is made of contiguous runs of 2^c amplitudes.  Consecutive segments k,
// k+1 therefore share c spins X_k ("exit set" of k): sweep k writes its tile
// back with X_k moved into the low bits (an in-place relabelling of bit
// positions inside the tile), and segment k+1 is grown starting from X_k.
// On the way back (reverse half step) each sweep undoes its relabelling, so
// the layout at every step boundary is the same (pos).
#include <algorithm>
#include <array>
#include <limits>
#include <queue>

#include "internal.h"

namespace spinrp {

namespace {

struct Frontier {
  const std::vector<std::pair<int, int>> *bonds;
  const std::vector<std::vector<int>> *chain;  // per spin: bonds touching it, in order
  std::vector<int> ptr;                        // per spin: next undone position in its chain
  int ndone = 0;

  bool ready(int b) const {
    const auto &bd = (*bonds)[b];
    const auto &ci = (*chain)[bd.first], &cj = (*chain)[bd.second];
    return ptr[bd.first] < (int)ci.size() && ci[ptr[bd.first]] == b &&
           ptr[bd.second] < (int)cj.size() && cj[ptr[bd.second]] == b;
  }
  int head(int q) const {
    const auto &c = (*chain)[q];
    return ptr[q] < (int)c.size() ? c[ptr[q]] : -1;
  }
  int pending(int q) const { return (int)(*chain)[q].size() - ptr[q]; }
  // Apply every gate reachable inside spin set Q (bit mask), smallest bond
  // index first; appends the applied bonds to out (if non-null).
  int closure(uint64_t Q, std::vector<int> *out) {
    std::priority_queue<int, std::vector<int>, std::greater<int>> pq;
    const int M = (int)ptr.size();
    for (int q = 0; q < M; ++q) {
      if (!((Q >> q) & 1)) continue;
      int b = head(q);
      if (b < 0) continue;
      const auto &bd = (*bonds)[b];
      if (((Q >> bd.first) & 1) && ((Q >> bd.second) & 1) && ready(b)) pq.push(b);
    }
    int applied = 0, last = -1;
    while (!pq.empty()) {
      int b = pq.top();
      pq.pop();
      if (b == last || !ready(b)) continue;  // pushed once per endpoint
      last = b;
      const auto &bd = (*bonds)[b];
      ++ptr[bd.first];
      ++ptr[bd.second];
      ++applied;
      ++ndone;
      if (out) out->push_back(b);
      for (int q : {bd.first, bd.second}) {
        int nb = head(q);
        if (nb < 0) continue;
        const auto &nbd = (*bonds)[nb];
        if (((Q >> nbd.first) & 1) && ((Q >> nbd.second) & 1) && ready(nb)) pq.push(nb);
      }
    }
    return applied;
  }
};

}  // namespace

bool build_plan(int M, const std::vector<std::pair<int, int>> &bonds, int K, int c, Plan *plan,
                std::string *err) {
  if (M < 1 || M > kMaxM || K < 1) {
    *err = "plan: bad size";
    return false;
  }
  const int B = (int)bonds.size();
  plan->M = M;
  plan->seg.clear();
  plan->segQ.clear();
  plan->exitX.clear();
  plan->pos.assign(M, -1);
  if (K >= M) {
    // one tile holds the whole state: one segment, canonical order, identity layout
    plan->K = M;
    plan->c = M;
    std::vector<PlanGate> g;
    for (int b = 0; b < B; ++b) g.push_back({b, bonds[b].first, bonds[b].second});
    plan->seg.push_back(g);
    std::vector<int> all(M);
    for (int q = 0; q < M; ++q) all[q] = q, plan->pos[q] = q;
    plan->segQ.push_back(all);
    return true;
  }
  c = std::max(0, std::min(c, K - 2));
  plan->K = K;
  plan->c = c;

  std::vector<std::vector<int>> chain(M);
  for (int b = 0; b < B; ++b) {
    chain[bonds[b].first].push_back(b);
    chain[bonds[b].second].push_back(b);
  }
  Frontier fr;
  fr.bonds = &bonds;
  fr.chain = &chain;
  fr.ptr.assign(M, 0);

  std::vector<int> order;  // spins in order of first use (physical layout)
  uint64_t placed = 0;
  auto place = [&](int q) {
    if (!((placed >> q) & 1)) order.push_back(q), placed |= 1ull << q;
  };

  uint64_t entry = 0;  // spins the next segment must contain (previous exit set)
  int guard = 0;
  while (fr.ndone < B || plan->seg.empty()) {
    if (++guard > 4 * B + 8) {
      *err = "plan: no progress (tile too narrow)";
      return false;
    }
    uint64_t Q = entry;
    std::vector<int> added;
    while (__builtin_popcountll(Q) < K) {
      Frontier base_trial = fr;
      const long base = base_trial.closure(Q, nullptr);
      int best = -1;
      long best_gain = -1, best_adj = -1, best_first = std::numeric_limits<long>::min();
      for (int q = 0; q < M; ++q) {
        if ((Q >> q) & 1) continue;
        Frontier trial = fr;
        const long gain = trial.closure(Q | (1ull << q), nullptr);
        long adj = 0, first = B;
        for (int k = fr.ptr[q]; k < (int)chain[q].size(); ++k) {
          const int b = chain[q][k];
          const int other = bonds[b].first == q ? bonds[b].second : bonds[b].first;
          if ((Q >> other) & 1) ++adj;
          first = std::min<long>(first, b);
        }
        const bool better = best < 0 || gain > best_gain || (gain == best_gain && adj > best_adj) ||
                            (gain == best_gain && adj == best_adj && -first > best_first);
        if (better) best = q, best_gain = gain, best_adj = adj, best_first = -first;
      }
      if (best < 0) break;
      if (best_gain <= base) {
        // no single spin adds a gate: take the spins of the earliest gate that
        // is ready after the closure of Q and fits (the smallest undone gate is
        // always ready, so with K >= c + 2 this always makes progress)
        Frontier after = fr;
        after.closure(Q, nullptr);
        const int room = K - __builtin_popcountll(Q);
        int pick = -1;
        for (int b = 0; b < B && pick < 0; ++b) {
          if (!after.ready(b)) continue;
          const int need = !((Q >> bonds[b].first) & 1) + !((Q >> bonds[b].second) & 1);
          if (need > 0 && need <= room) pick = b;
        }
        if (pick < 0) break;
        for (int q : {bonds[pick].first, bonds[pick].second})
          if (!((Q >> q) & 1)) Q |= 1ull << q, added.push_back(q);
        continue;
      }
      Q |= 1ull << best;
      added.push_back(best);
    }
    // a tile always spans exactly K spins: pad with unused ones
    for (int q = 0; q < M && __builtin_popcountll(Q) < K; ++q)
      if (!((Q >> q) & 1)) Q |= 1ull << q, added.push_back(q);
    std::vector<int> applied;
    fr.closure(Q, &applied);
    if (applied.empty() && fr.ndone < B) {
      *err = "plan: a segment placed no gate (tile too narrow)";
      return false;
    }
    std::vector<PlanGate> g;
    for (int b : applied) g.push_back({b, bonds[b].first, bonds[b].second});
    plan->seg.push_back(g);
    std::vector<int> qs;
    for (int q = 0; q < M; ++q)
      if ((Q >> q) & 1) qs.push_back(q);
    plan->segQ.push_back(qs);
    // exit set: the c spins of Q whose next pending gate comes earliest
    std::vector<std::pair<long, int>> cand;
    for (int q : qs) {
      const int h = fr.head(q);
      cand.push_back({h < 0 ? (long)B + 1000 - fr.pending(q) : (long)h, q});
    }
    std::sort(cand.begin(), cand.end());
    std::vector<int> X;
    for (int k = 0; k < c; ++k) X.push_back(cand[k].second);
    std::sort(X.begin(), X.end());
    plan->exitX.push_back(X);
    entry = 0;
    for (int q : X) entry |= 1ull << q;
    for (int q : added) place(q);
  }
  const int s = (int)plan->seg.size();
  // layout at step boundaries: the first exit set in the low bits (for a
  // single segment: the first c spins of its tile), then spins in order of use
  std::vector<int> low = s >= 2 ? plan->exitX[0]
                                : std::vector<int>(plan->segQ[0].begin(), plan->segQ[0].begin() + c);
  std::vector<int> final_order = low;
  uint64_t in_low = 0;
  for (int q : low) in_low |= 1ull << q;
  for (int q : order)
    if (!((in_low >> q) & 1)) final_order.push_back(q);
  for (int q = 0; q < M; ++q)
    if (!((placed >> q) & 1) && !((in_low >> q) & 1)) final_order.push_back(q);
  for (int p = 0; p < M; ++p) plan->pos[final_order[p]] = p;
  plan->exitX.resize(std::max(0, s - 1));
  return true;
}


// ---------------------------------------------------------------------------
// Phases of the register-blocked sweep: the gates of a pass (on its K tile
// bits) are applied in phases, each holding RB tile bits in registers.  A
// phase applies every gate both of whose bits it holds as soon as all earlier
// gates on those bits are done (so each bit keeps its gate sequence and the
// operator is unchanged).  Fewer phases mean fewer shared-memory round trips;
// a beam search over the register sets looks further ahead than the greedy
// segment planner.
// ---------------------------------------------------------------------------
namespace {

typedef std::array<uint8_t, kMaxK> BitPtr;  // per tile bit: gates of its chain done

struct PhaseState {
  BitPtr ptr;
  int done = 0;
  int pre = 0;               // gates before the fence done
  int parent = -1;           // index into the previous beam level
  uint32_t set = 0;          // register set that produced this state
};

// Apply every gate reachable inside bit set R (smallest index first); gates
// from `fence` on only once every gate before it is done (*pre counts those).
int phase_closure(const std::vector<std::pair<int, int>> &g, const std::vector<std::vector<int>> &chain,
                  BitPtr &ptr, uint32_t R, int fence, int *pre, std::vector<int> *out) {
  auto ready = [&](int b) {
    const int u = g[b].first, v = g[b].second;
    return (b < fence || *pre == fence) && ptr[u] < chain[u].size() && chain[u][ptr[u]] == b &&
           ptr[v] < chain[v].size() && chain[v][ptr[v]] == b;
  };
  int applied = 0;
  for (bool progress = true; progress;) {
    progress = false;
    int best = -1;
    for (int q = 0; q < (int)chain.size(); ++q) {
      if (!((R >> q) & 1) || ptr[q] >= chain[q].size()) continue;
      const int b = chain[q][ptr[q]];
      if (((R >> g[b].first) & 1) && ((R >> g[b].second) & 1) && ready(b) && (best < 0 || b < best)) best = b;
    }
    if (best >= 0) {
      ++ptr[g[best].first];
      ++ptr[g[best].second];
      ++applied;
      if (best < fence) ++*pre;
      if (out) out->push_back(best);
      progress = true;
    }
  }
  return applied;
}

}  // namespace

// Every combination of `take` out of the n items (indices), in lexicographic
// order, passed to f as a bit mask over items[].
template <typename F>
static void for_each_subset(const std::vector<int> &items, int take, F f) {
  const int n = (int)items.size();
  if (take > n || take < 0) return;
  std::vector<int> pick(take);
  for (int i = 0; i < take; ++i) pick[i] = i;
  while (true) {
    uint32_t R = 0;
    for (int i : pick) R |= 1u << items[i];
    f(R);
    int i = take - 1;
    while (i >= 0 && pick[i] == n - take + i) --i;
    if (i < 0) break;
    ++pick[i];
    for (int j = i + 1; j < take; ++j) pick[j] = pick[j - 1] + 1;
  }
}

bool plan_phases(int K, const std::vector<std::pair<int, int>> &gates, int RB, int beam, int fence,
                 std::vector<uint32_t> *sets, std::vector<std::vector<int>> *applied, uint32_t black,
                 uint32_t nb_allowed) {
  sets->clear();
  applied->clear();
  const int n = (int)gates.size();
  if (n == 0) return true;
  std::vector<std::vector<int>> chain(K);
  for (int b = 0; b < n; ++b) {
    if (gates[b].first < 0 || gates[b].first >= K || gates[b].second < 0 || gates[b].second >= K ||
        gates[b].first == gates[b].second)
      return false;
    chain[gates[b].first].push_back(b);
    chain[gates[b].second].push_back(b);
  }
  std::vector<std::vector<PhaseState>> levels(1);
  if (fence < 0 || fence > n) fence = n;
  BitPtr zero;
  zero.fill(0);
  levels[0].push_back(PhaseState{zero, 0, 0, -1, 0});
  for (int depth = 0; depth < 4 * n + 4; ++depth) {
    const std::vector<PhaseState> &cur = levels.back();
    std::vector<PhaseState> next;
    for (int si = 0; si < (int)cur.size(); ++si) {
      const PhaseState &st = cur[si];
      // bits with gates still to do; a useful set holds RB of them (all of
      // them when fewer remain), padded with idle bits
      std::vector<int> live;
      for (int q = 0; q < K; ++q)
        if (st.ptr[q] < chain[q].size()) live.push_back(q);
      auto try_set = [&](uint32_t R) {
        PhaseState ch{st.ptr, st.done, st.pre, si, R};
        const int a = phase_closure(gates, chain, ch.ptr, R, fence, &ch.pre, nullptr);
        if (a > 0) {
          ch.done += a;
          next.push_back(std::move(ch));
        }
      };
      if (nb_allowed == 0) {
        const int take = std::min<int>(RB, (int)live.size());
        for_each_subset(live, take, [&](uint32_t R) {
          for (int q = 0; q < K && __builtin_popcount(R) < RB; ++q) R |= 1u << q;
          try_set(R);
        });
      } else {
        // for each allowed count nb: nb live bits of the colour `black` and
        // RB - nb of the other (fewer when fewer are live), each side padded
        // with idle bits of its colour
        std::vector<int> lb, lw;
        for (int q : live) (((black >> q) & 1u) ? lb : lw).push_back(q);
        for (int nb = 0; nb <= RB; ++nb) {
          if (!((nb_allowed >> nb) & 1u)) continue;
          const int tb = std::min<int>(nb, (int)lb.size()), tw = std::min<int>(RB - nb, (int)lw.size());
          for_each_subset(lb, tb, [&](uint32_t Rb) {
            for (int q = 0; q < K && __builtin_popcount(Rb) < nb; ++q)
              if ((black >> q) & 1u) Rb |= 1u << q;
            if (__builtin_popcount(Rb) != nb) return;
            for_each_subset(lw, tw, [&](uint32_t Rw) {
              for (int q = 0; q < K && __builtin_popcount(Rw) < RB - nb; ++q)
                if (!((black >> q) & 1u)) Rw |= 1u << q;
              if (__builtin_popcount(Rw) != RB - nb) return;
              try_set(Rb | Rw);
            });
          });
        }
      }
    }
    if (next.empty()) return false;
    // keep the `beam` best distinct states (most gates done)
    std::stable_sort(next.begin(), next.end(),
                     [](const PhaseState &a, const PhaseState &b) { return a.done > b.done; });
    std::vector<PhaseState> kept;
    for (PhaseState &c : next) {
      bool dup = false;
      for (const PhaseState &k : kept)
        if (k.ptr == c.ptr) {
          dup = true;
          break;
        }
      if (!dup) kept.push_back(std::move(c));
      if ((int)kept.size() >= beam) break;
    }
    levels.push_back(std::move(kept));
    if (levels.back().front().done == n) {
      // walk back the sets of the first finished state, then replay them
      std::vector<uint32_t> path;
      for (int lv = (int)levels.size() - 1, si = 0; lv > 0; --lv) {
        path.push_back(levels[lv][si].set);
        si = levels[lv][si].parent;
      }
      std::reverse(path.begin(), path.end());
      BitPtr ptr = zero;
      int pre = 0;
      for (uint32_t R : path) {
        std::vector<int> out;
        phase_closure(gates, chain, ptr, R, fence, &pre, &out);
        sets->push_back(R);
        applied->push_back(out);
      }
      return true;
    }
  }
  return false;
}

}  // namespace spinrp
