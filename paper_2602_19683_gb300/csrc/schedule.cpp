// Task graphs of the tiled algorithms (Sec. 3.2, Fig. 1; Eqs. 2-3) and a list scheduler that orders
// them for the persistent kernel. The paper's runtime fires a task when the futures of its input
// tiles resolve (HPX dataflow, Sec. 2.1); here the same dependencies are resolved on the device by
// per-tile counters, and the host only chooses the order in which CTAs pick tasks up.
#include "schedule.h"

#include <algorithm>
#include <queue>
#include <unordered_map>
#include <utility>

#include "kernels.h"

namespace gpk {

std::vector<int> list_schedule(const std::vector<double>& cost, const std::vector<std::vector<int>>& preds,
                               int workers, const std::vector<double>* group_key, const LocalityKeys* loc) {
  const int n = (int)cost.size();
  std::vector<std::vector<int>> succ(n);
  std::vector<int> indeg(n, 0);
  for (int t = 0; t < n; ++t) {
    indeg[t] = (int)preds[t].size();
    for (int p : preds[t]) succ[p].push_back(t);
  }
  // Bottom level: longest cost path from a task to the end. Tasks are created in a topological
  // order (every predecessor has a smaller index), so one backward sweep suffices.
  std::vector<double> bl(n, 0.0);
  for (int t = n - 1; t >= 0; --t) {
    double m = 0.0;
    for (int s : succ[t]) m = std::max(m, bl[s]);
    bl[t] = cost[t] + m;
  }
  auto cmp = [&](int a, int b) {
    if (group_key && (*group_key)[a] != (*group_key)[b]) return (*group_key)[a] < (*group_key)[b];
    return bl[a] < bl[b] || (bl[a] == bl[b] && a > b);
  };
  std::priority_queue<int, std::vector<int>, decltype(cmp)> ready(cmp);
  // operand locality: ready tasks by key (entries of started tasks are dropped lazily)
  const bool use_loc = loc && loc->eps > 0 && (int)loc->a.size() == n && (int)loc->b.size() == n;
  std::unordered_map<long long, std::vector<int>> by_a, by_b;
  std::vector<char> started(n, 0);
  long long last_a = -1, last_b = -1;
  auto make_ready = [&](int t) {
    ready.push(t);
    if (use_loc) {
      if (loc->a[t] >= 0) by_a[loc->a[t]].push_back(t);
      if (loc->b[t] >= 0) by_b[loc->b[t]].push_back(t);
    }
  };
  // the best-ranked ready task sharing key k (or -1), dropping started ones from the list
  auto best_sharing = [&](std::unordered_map<long long, std::vector<int>>& m, long long k, int best) {
    if (k < 0) return best;
    auto it = m.find(k);
    if (it == m.end()) return best;
    std::vector<int>& v = it->second;
    size_t w = 0;
    for (size_t i = 0; i < v.size(); ++i)
      if (!started[v[i]]) v[w++] = v[i];
    v.resize(w);
    for (int c : v)
      if (best < 0 || bl[c] > bl[best]) best = c;
    return best;
  };
  for (int t = 0; t < n; ++t)
    if (indeg[t] == 0) make_ready(t);
  using Ev = std::pair<double, int>;  // (finish time, task)
  std::priority_queue<Ev, std::vector<Ev>, std::greater<Ev>> running;
  std::vector<int> order;
  order.reserve(n);
  double now = 0.0;
  int free_workers = std::max(1, workers);
  while ((int)order.size() < n) {
    while (free_workers > 0) {
      while (!ready.empty() && started[ready.top()]) ready.pop();
      if (ready.empty()) break;
      int t = ready.top();
      if (use_loc) {
        const int c = best_sharing(by_b, last_b, best_sharing(by_a, last_a, -1));
        if (c >= 0 && bl[c] >= (1.0 - loc->eps) * bl[t]) t = c;
        if (loc->a[t] >= 0) last_a = loc->a[t];
        if (loc->b[t] >= 0) last_b = loc->b[t];
      }
      if (t == ready.top()) ready.pop();
      started[t] = 1;
      order.push_back(t);
      running.push({now + cost[t], t});
      --free_workers;
    }
    if (running.empty()) break;  // cannot happen for a DAG
    const Ev e = running.top();
    running.pop();
    now = e.first;
    ++free_workers;
    for (int s : succ[e.second])
      if (--indeg[s] == 0) make_ready(s);
  }
  return order;
}

namespace {

struct Builder {
  std::vector<Task4> tasks;
  std::vector<double> cost;
  std::vector<std::vector<int>> preds;
  int add(int kind, int p, int q, int r, double c, std::initializer_list<int> deps) {
    return add_v(kind, p, q, r, c, std::vector<int>(deps));
  }
  int add_v(int kind, int p, int q, int r, double c, const std::vector<int>& deps) {
    tasks.push_back({kind, p, q, r});
    cost.push_back(c);
    std::vector<int> d;
    for (int x : deps)
      if (x >= 0) d.push_back(x);
    preds.push_back(std::move(d));
    return (int)tasks.size() - 1;
  }
  std::vector<Task4> ordered(int workers, const std::vector<double>* group_key = nullptr,
                             const LocalityKeys* loc = nullptr) const {
    std::vector<int> ord = list_schedule(cost, preds, workers, group_key, loc);
    std::vector<Task4> out;
    out.reserve(ord.size());
    for (int t : ord) out.push_back(tasks[t]);
    return out;
  }
};

inline size_t tri(int I, int J) { return (size_t)I * (I + 1) / 2 + J; }

}  // namespace

std::vector<Task4> cholesky_tasks(int Mt, int T, int workers, const CostModel& cm) {
  Builder b;
  const double t3 = (double)T * T * T;
  const double spf_upd = cm.mixed ? cm.sec_per_flop32 : cm.sec_per_flop;
  double c_potrf = cm.task_overhead + cm.sec_per_flop * t3 / 3.0 / cm.potrf_eff;
  double c_trsm0 = cm.task_overhead + cm.sec_per_flop * t3 / cm.trsm_eff;
  double c_trsm = cm.task_overhead + spf_upd * t3 / cm.trsm_eff;
  double c_gemm = cm.task_overhead + spf_upd * 2.0 * t3 / cm.gemm_eff;
  double c_syrk = cm.task_overhead + spf_upd * (t3 + 64.0 * T * T) / cm.gemm_eff;
  if (cm.tensor_cores) {  // measured at T = 128: POTRF + FP32 inverse 403 us, FP64 TRSM 440 us, tensor
                          // TRSM 30 us, one column pair of a grouped update 6.6 us (5 us on the diagonal)
    const double s3 = t3 / (128.0 * 128.0 * 128.0), s2 = (double)T * T / (128.0 * 128.0);
    c_potrf = cm.tc_potrf * s3;
    c_trsm0 = cm.tc_trsm0 * s3;
    c_trsm = cm.tc_trsm * s2;
    c_gemm = cm.tc_gemm * s2;
    c_syrk = cm.tc_syrk * s2;
  }
  if (cm.variant == 1 || cm.variant == 2) {
    // left-/top-looking: tile (I, K) takes all its updates (columns J < K) in one task, then its
    // POTRF / TRSM; dispatched in column order (left) or row order (top), longest path within
    std::vector<int> fin(tri(Mt, 0), -1);  // the task that made tile (I, K) final
    std::vector<double> key;
    auto keyed = [&](int t, double k) {
      if ((int)key.size() <= t) key.resize(t + 1, 0.0);
      key[t] = k;
    };
    const bool left = cm.variant == 1;
    for (int a = 0; a < Mt; ++a)          // left: a = column K, c = row I >= K; top: a = row I, c = column K <= I
      for (int c = left ? a : 0; left ? c < Mt : c <= a; ++c) {
        const int I = left ? c : a, K = left ? a : c;
        std::vector<int> deps;
        int upd = -1;
        if (K > 0) {
          for (int J = 0; J < K; ++J) {
            deps.push_back(fin[tri(I, J)]);
            deps.push_back(fin[tri(K, J)]);
          }
          upd = b.add_v(TASK_UPD, I, K, 0 | (K << 16), K * (I == K ? c_syrk : c_gemm), deps);
          keyed(upd, -(double)a);
        }
        int t;
        if (I == K) {
          t = b.add(TASK_POTRF, K, 0, 0, c_potrf, {upd});
          keyed(t, -(double)a);
          keyed(b.add(TASK_TRTRI, K, 0, 0, c_trsm0, {t}), -(double)a);
        } else {
          t = b.add(TASK_TRSM, I, K, 0, K == 0 ? c_trsm0 : c_trsm, {fin[tri(K, K)], upd});
          keyed(t, -(double)a);
        }
        fin[tri(I, K)] = t;
      }
    key.resize(b.tasks.size(), 0.0);
    return b.ordered(workers, &key);
  }
  // Updates of a tile whose critical use is still far away are grouped: columns [J0, J1) in one task
  // (one pass over the tile's C instead of J1 - J0); the last kTail columns before the tile is needed
  // stay single so the critical path is not lengthened.
  const int g = cm.update_group > 1 ? cm.update_group : 1;
  const int kTail = 2;
  std::vector<int> last(tri(Mt, 0), -1);  // last task that wrote each lower tile
  std::vector<int> gstart(tri(Mt, 0), 0);  // first column of the open update group of each tile
  std::vector<int> trsm_of(tri(Mt, 0), -1);
  for (int J = 0; J < Mt; ++J) {
    const int po = b.add(TASK_POTRF, J, 0, 0, c_potrf, {last[tri(J, J)]});
    last[tri(J, J)] = po;
    b.add(TASK_TRTRI, J, 0, 0, c_trsm0, {po});  // inverse of L_JJ for the vector solves; nothing waits on it
    for (int I = J + 1; I < Mt; ++I) {
      last[tri(I, J)] = b.add(TASK_TRSM, I, J, 0, J == 0 ? c_trsm0 : c_trsm, {po, last[tri(I, J)]});
      trsm_of[tri(I, J)] = last[tri(I, J)];
    }
    for (int K = J + 1; K < Mt; ++K) {
      const int lim = K - kTail;  // columns >= lim are applied one by one
      const bool grouped = g > 1 && J < lim;
      // group boundaries depend on the column K only, so every row of column K closes its group here
      if (grouped && (J + 1) % g != 0 && J + 1 != lim) continue;  // the group stays open
      for (int I = K; I < Mt; ++I) {
        const size_t t = tri(I, K);
        const int J0 = grouped ? gstart[t] : J;
        // rows K, K+1 | K+2, K+3 | ... of a closing group share one pass over L_KJ
        const bool pair = grouped && cm.pair_rows && (I - K) % 2 == 0 && I + 1 < Mt;
        std::vector<int> deps{last[t]};
        if (pair) deps.push_back(last[tri(I + 1, K)]);
        for (int Jj = J0; Jj <= J; ++Jj) {
          deps.push_back(trsm_of[tri(I, Jj)]);
          if (pair) deps.push_back(trsm_of[tri(I + 1, Jj)]);
          deps.push_back(trsm_of[tri(K, Jj)]);
        }
        const int r = J0 | ((J + 1) << 16);
        const double cost = (J + 1 - J0) * (I == K ? c_syrk : c_gemm);
        if (pair) {
          // measured at n = 32768: about as long as the two tiles' separate tasks (97 us for ~2 x 7
          // column pairs: the L2 already served the shared L_KJ to neighbouring tasks); ranking it at
          // 0.8 of that gave the shorter factorisation of the two weights tried (152 vs 156 ms)
          const int id = b.add_v(TASK_UPD2, I, K, r, 0.8 * (cost + (J + 1 - J0) * c_gemm), deps);
          last[t] = last[tri(I + 1, K)] = id;
          gstart[t] = gstart[tri(I + 1, K)] = J + 1;
          ++I;
        } else {
          last[t] = b.add_v(TASK_UPD, I, K, r, cost, deps);
          gstart[t] = J + 1;
        }
      }
    }
  }
  // Longest-remaining-path order. (A column-group / super-tile order for the grouped updates keeps
  // their operands in L2 — 98 % modelled hits against 14 % — but delays the updates the diagonal
  // chain waits for; measured at n = 32768 both orders give the same factorisation time.) With
  // cm.locality_eps, grouped updates that share a packed operand group -- L_{I,J0..J1} (a) or
  // L_{K,J0..J1} (b) -- are started back to back when their rank allows (LocalityKeys).
  if (cm.locality_eps <= 0.0) return b.ordered(workers);
  LocalityKeys loc;
  loc.eps = cm.locality_eps;
  loc.a.assign(b.tasks.size(), -1);
  loc.b.assign(b.tasks.size(), -1);
  for (size_t i = 0; i < b.tasks.size(); ++i) {
    const Task4& t = b.tasks[i];
    const int J0 = t.r & 0xFFFF, J1 = t.r >> 16;
    if ((t.kind == TASK_UPD || t.kind == TASK_UPD2) && J1 - J0 > 1) {
      loc.a[i] = (long long)t.p * 65536 + J0;
      loc.b[i] = (long long)t.q * 65536 + J0;
    }
  }
  return b.ordered(workers, nullptr, &loc);
}

std::vector<Task4> cov_tasks(int Mt, int Mc, int T, int workers, const CostModel& cm, bool with_w) {
  Builder b;
  const double t3 = (double)T * T * T;
  const double spf = cm.mixed ? cm.sec_per_flop32 : cm.sec_per_flop;
  double c_trsm = cm.task_overhead + spf * t3 / cm.trsm_eff;
  double c_gemm = cm.task_overhead + spf * 2.0 * t3 / cm.gemm_eff;
  if (cm.tensor_cores) {  // measured at T = 128: V solve 35 us, one column pair of a grouped product 5.5 us
    const double s2 = (double)T * T / (128.0 * 128.0);
    c_trsm = cm.tc_vtrsm * s2;
    c_gemm = cm.tc_vgemm * s2;
  }
  // Mixed mode on the tensor cores groups the products into one output tile: V_Ic takes columns
  // [J0, J1) together while they are far from its own solve (the last kTail one by one, as they
  // gate the solve chain); S_ab takes every g consecutive J together.
  const int g = cm.update_group > 1 ? cm.update_group : 1;
  const int kTail = 2;
  std::vector<int> lastV((size_t)Mt * Mc, -1), lastS(tri(Mc, 0), -1), vtrsm((size_t)Mt * Mc, -1);
  std::vector<int> gstartV((size_t)Mt * Mc, 0), gstartS(tri(Mc, 0), 0);
  // With grouped products: the solve chain (V solves and the single products next to them) first;
  // the grouped products after it in column-group order, then by block row I and column block c, so
  // that consecutive products share the L panel tiles of row I and the group's V blocks stay in L2.
  std::vector<double> key;
  auto keyed = [&](int t, double k) {
    if (g == 1) return;
    if ((int)key.size() <= t) key.resize(t + 1, 1.0);
    key[t] = k;
  };
  const double grp = (double)Mt * Mc + 1.0;
  for (int J = 0; J < Mt; ++J) {
    for (int c = 0; c < Mc; ++c) {
      lastV[(size_t)J * Mc + c] = b.add(TASK_VTRSM, J, c, 0, c_trsm, {lastV[(size_t)J * Mc + c]});
      vtrsm[(size_t)J * Mc + c] = lastV[(size_t)J * Mc + c];
      keyed(vtrsm[(size_t)J * Mc + c], 1.0);
    }
    for (int I = J + 1; I < Mt; ++I)
      for (int c = 0; c < Mc; ++c) {
        const size_t v = (size_t)I * Mc + c;
        if (g == 1) {
          lastV[v] = b.add(TASK_VGEMM, I, J, c, c_gemm, {vtrsm[(size_t)J * Mc + c], lastV[v]});
          continue;
        }
        const int lim = I - kTail;
        int J0 = J;
        if (J < lim) {
          if ((J + 1) % g != 0 && J + 1 != lim) continue;  // the group stays open
          J0 = gstartV[v];
        }
        std::vector<int> deps{lastV[v]};
        for (int Jj = J0; Jj <= J; ++Jj) deps.push_back(vtrsm[(size_t)Jj * Mc + c]);
        lastV[v] = b.add_v(TASK_VGEMM_G, I, c, J0 | ((J + 1) << 16), (J + 1 - J0) * c_gemm, deps);
        gstartV[v] = J + 1;
        keyed(lastV[v], J < lim ? -((double)(J0 / g) * grp + (double)I * Mc + c) - 1.0 : 1.0);
      }
    if (!with_w) continue;  // variance only: V is all that is needed
    for (int a = 0; a < Mc; ++a)
      for (int bb = 0; bb <= a; ++bb) {
        const size_t sidx = tri(a, bb);
        if (g == 1) {
          lastS[sidx] = b.add(TASK_WSYRK, a, bb, J, c_gemm,
                              {vtrsm[(size_t)J * Mc + a], vtrsm[(size_t)J * Mc + bb], lastS[sidx]});
          continue;
        }
        if ((J + 1) % g != 0 && J + 1 != Mt) continue;
        const int J0 = gstartS[sidx];
        std::vector<int> deps{lastS[sidx]};
        for (int Jj = J0; Jj <= J; ++Jj) {
          deps.push_back(vtrsm[(size_t)Jj * Mc + a]);
          deps.push_back(vtrsm[(size_t)Jj * Mc + bb]);
        }
        lastS[sidx] = b.add_v(TASK_WSYRK_G, a, bb, J0 | ((J + 1) << 16), (J + 1 - J0) * c_gemm, deps);
        gstartS[sidx] = J + 1;
        keyed(lastS[sidx], -((double)(J0 / g) * grp + (double)Mt * Mc) - 1.0);
      }
  }
  if (g == 1) return b.ordered(workers);
  key.resize(b.tasks.size(), 1.0);
  return b.ordered(workers, &key);
}

// Reverse of Fig. 1's algorithm for the adjoint Lbar -> Abar: for J = Mt-1 down to 0, first undo
// step J's trailing updates (RUPD: Lbar_PJ -= Abar~_PK L_KJ for every P, K > J, K ascending), then
// its TRSMs (RTRSM: Abar_PJ = Lbar_PJ L_JJ^{-1}, and RDIAG: Lbar_JJ -= tril(Abar_PJ^T L_PJ)), then
// its POTRF (RPOTRF).
std::vector<Task4> cholesky_adjoint_tasks(int Mt, int T, int workers, const CostModel& cm) {
  Builder b;
  const double t3 = (double)T * T * T;
  const double spf_upd = cm.mixed ? cm.sec_per_flop32 : cm.sec_per_flop;
  const double c_rupd = cm.task_overhead + spf_upd * 2.0 * t3 / cm.gemm_eff;
  const double c_rtrsm = cm.task_overhead + cm.sec_per_flop * t3 / cm.trsm_eff;
  const double c_rdiag = cm.task_overhead + spf_upd * 2.0 * t3 / cm.gemm_eff;
  const double c_rpotrf = cm.task_overhead + cm.sec_per_flop * 3.0 * t3 / cm.trsm_eff;
  std::vector<int> last(tri(Mt, 0), -1);   // last writer of Lbar/Abar of each lower tile
  std::vector<int> final_(tri(Mt, 0), -1);  // task that made Abar of the tile final
  std::vector<int> lastpart(kAdjParts, -1);
  for (int J = Mt - 1; J >= 0; --J) {
    // Lbar_PJ accumulates its terms with K descending: the K = J+1 term, the last to become
    // available, is applied last, so the others run ahead.
    for (int P = J + 1; P < Mt; ++P)
      for (int K = Mt - 1; K > J; --K) {
        const int hi = P > K ? P : K, lo = P > K ? K : P;
        last[tri(P, J)] = b.add(TASK_RUPD, P, K, J, c_rupd, {final_[tri(hi, lo)], last[tri(P, J)]});
      }
    for (int P = J + 1; P < Mt; ++P) {
      const int t = b.add(TASK_RTRSM, P, J, 0, c_rtrsm, {last[tri(P, J)]});
      last[tri(P, J)] = t;
      final_[tri(P, J)] = t;
    }
    // the diagonal adjoint's contributions go to kAdjParts partial sums (P - J - 1 mod kAdjParts)
    for (int q = 0; q < kAdjParts; ++q) lastpart[q] = -1;
    for (int P = J + 1; P < Mt; ++P) {
      const int q = (P - J - 1) % kAdjParts;
      lastpart[q] = b.add(TASK_RDIAG, P, J, 0, c_rdiag, {final_[tri(P, J)], lastpart[q]});
    }
    std::vector<int> deps(lastpart.begin(), lastpart.end());
    b.tasks.push_back({TASK_RPOTRF, J, 0, 0});
    b.cost.push_back(c_rpotrf);
    std::vector<int> pr;
    for (int x : deps)
      if (x >= 0) pr.push_back(x);
    b.preds.push_back(pr);
    const int t = (int)b.tasks.size() - 1;
    last[tri(J, J)] = t;
    final_[tri(J, J)] = t;
  }
  return b.ordered(workers);
}

namespace {

// Appends GP g's Cholesky, mean-solve and (optionally) covariance tasks, with the cross-graph
// dependencies on the factor tiles.
void append_gp(Builder& b, int g, const BatchGp& gp, bool want_cov, const CostModel& cm) {
  const int Mt = gp.Mt, Mc = gp.Mc, T = gp.T, nch = T / 32;
  const int tag = g << kBatchKindBits;
  const double t3 = (double)T * T * T;
  const double spf = cm.mixed ? cm.sec_per_flop32 : cm.sec_per_flop;
  const double c_potrf = cm.task_overhead + cm.sec_per_flop * t3 / 3.0 / cm.potrf_eff;
  const double c_trsm = cm.task_overhead + spf * t3 / cm.trsm_eff;
  const double c_gemm = cm.task_overhead + spf * 2.0 * t3 / cm.gemm_eff;
  const double c_solve = cm.task_overhead + cm.sec_per_flop * (double)T * T / cm.vec_eff;
  const double c_gemv = cm.task_overhead + cm.sec_per_flop * 2.0 * 32.0 * T / cm.vec_eff;
  std::vector<int> last(tri(Mt, 0), -1);
  for (int J = 0; J < Mt; ++J) {
    const int po = b.add(TASK_POTRF | tag, J, 0, 0, c_potrf, {last[tri(J, J)]});
    last[tri(J, J)] = po;
    for (int I = J + 1; I < Mt; ++I) last[tri(I, J)] = b.add(TASK_TRSM | tag, I, J, 0, c_trsm, {po, last[tri(I, J)]});
    for (int I = J + 1; I < Mt; ++I)
      for (int K = J + 1; K <= I; ++K)
        last[tri(I, K)] = b.add(TASK_UPD | tag, I, K, J, c_gemm, {last[tri(I, J)], last[tri(K, J)], last[tri(I, K)]});
  }
  // last[] now holds the task that made each factor tile final
  std::vector<int> lastF((size_t)Mt * nch, -1), lastB((size_t)Mt * nch, -1), fsolve(Mt, -1);
  for (int J = 0; J < Mt; ++J) {
    b.tasks.push_back({TASK_FSOLVE | tag, J, 0, 0});
    b.cost.push_back(c_solve);
    std::vector<int> pr{last[tri(J, J)]};
    for (int ch = 0; ch < nch; ++ch)
      if (lastF[(size_t)J * nch + ch] >= 0) pr.push_back(lastF[(size_t)J * nch + ch]);
    b.preds.push_back(pr);
    fsolve[J] = (int)b.tasks.size() - 1;
    for (int I = J + 1; I < Mt; ++I)
      for (int ch = 0; ch < nch; ++ch)
        lastF[(size_t)I * nch + ch] =
            b.add(TASK_FGEMV | tag, I, J, ch, c_gemv, {fsolve[J], last[tri(I, J)], lastF[(size_t)I * nch + ch]});
  }
  for (int I = Mt - 1; I >= 0; --I) {
    b.tasks.push_back({TASK_BSOLVE | tag, I, 0, 0});
    b.cost.push_back(c_solve);
    std::vector<int> pr{fsolve[I]};
    for (int ch = 0; ch < nch; ++ch)
      if (lastB[(size_t)I * nch + ch] >= 0) pr.push_back(lastB[(size_t)I * nch + ch]);
    b.preds.push_back(pr);
    const int bs = (int)b.tasks.size() - 1;
    for (int J = 0; J < I; ++J)
      for (int ch = 0; ch < nch; ++ch)
        lastB[(size_t)J * nch + ch] =
            b.add(TASK_BGEMV | tag, J, I, ch, c_gemv, {bs, fsolve[J], last[tri(I, J)], lastB[(size_t)J * nch + ch]});
  }
  if (!want_cov) return;
  std::vector<int> lastV((size_t)Mt * Mc, -1), lastS(tri(Mc, 0), -1);
  for (int J = 0; J < Mt; ++J) {
    for (int c = 0; c < Mc; ++c)
      lastV[(size_t)J * Mc + c] = b.add(TASK_VTRSM | tag, J, c, 0, c_trsm, {last[tri(J, J)], lastV[(size_t)J * Mc + c]});
    for (int I = J + 1; I < Mt; ++I)
      for (int c = 0; c < Mc; ++c)
        lastV[(size_t)I * Mc + c] = b.add(TASK_VGEMM | tag, I, J, c, c_gemm,
                                          {last[tri(I, J)], lastV[(size_t)J * Mc + c], lastV[(size_t)I * Mc + c]});
    for (int a = 0; a < Mc; ++a)
      for (int bb = 0; bb <= a; ++bb)
        lastS[tri(a, bb)] = b.add(TASK_WSYRK | tag, a, bb, J, c_gemm,
                                  {lastV[(size_t)J * Mc + a], lastV[(size_t)J * Mc + bb], lastS[tri(a, bb)]});
  }
}

}  // namespace

std::vector<Task4> batch_tasks(const std::vector<BatchGp>& gps, bool want_cov, int workers, const CostModel& cm,
                               int order) {
  Builder b;
  std::vector<size_t> first(gps.size() + 1, 0);
  for (size_t g = 0; g < gps.size(); ++g) {
    first[g] = b.tasks.size();
    append_gp(b, (int)g, gps[g], want_cov, cm);
  }
  first[gps.size()] = b.tasks.size();
  if (order != 1) return b.ordered(workers);
  std::vector<double> key(b.tasks.size(), 0.0);  // each task carries its GP's total modelled work
  for (size_t g = 0; g < gps.size(); ++g) {
    double w = 0.0;
    for (size_t t = first[g]; t < first[g + 1]; ++t) w += b.cost[t];
    for (size_t t = first[g]; t < first[g + 1]; ++t) key[t] = w;
  }
  return b.ordered(workers, &key);
}

std::vector<Task4> mean_tasks(int Mt, int T, int workers, const CostModel& cm) {
  Builder b;
  const int nch = T / 32;
  // Each diagonal block is solved as nch 32-row chunks in parallel (products with the stored inverse
  // of the diagonal tile); the updates of the blocks further down are 32-row GEMV chunks.
  const double c_solve = cm.task_overhead + cm.sec_per_flop * 2.0 * 32.0 * T / cm.vec_eff;
  const double c_gemv = cm.task_overhead + cm.sec_per_flop * 2.0 * 32.0 * T / cm.vec_eff;
  std::vector<int> lastF((size_t)Mt * nch, -1), lastB((size_t)Mt * nch, -1);
  std::vector<std::vector<int>> fsolve(Mt), bsolve(Mt);
  for (int J = 0; J < Mt; ++J) {
    std::vector<int> pr;
    for (int ch = 0; ch < nch; ++ch) pr.push_back(lastF[(size_t)J * nch + ch]);
    for (int ch = 0; ch < nch; ++ch) fsolve[J].push_back(b.add_v(TASK_FSOLVE_C, J, ch, 0, c_solve, pr));
    for (int I = J + 1; I < Mt; ++I)
      for (int ch = 0; ch < nch; ++ch) {
        std::vector<int> d(fsolve[J]);
        d.push_back(lastF[(size_t)I * nch + ch]);
        lastF[(size_t)I * nch + ch] = b.add_v(TASK_FGEMV, I, J, ch, c_gemv, d);
      }
  }
  for (int I = Mt - 1; I >= 0; --I) {
    std::vector<int> pr(fsolve[I]);
    for (int ch = 0; ch < nch; ++ch) pr.push_back(lastB[(size_t)I * nch + ch]);
    for (int ch = 0; ch < nch; ++ch) bsolve[I].push_back(b.add_v(TASK_BSOLVE_C, I, ch, 0, c_solve, pr));
    for (int J = 0; J < I; ++J)
      for (int ch = 0; ch < nch; ++ch) {
        std::vector<int> d(bsolve[I]);
        d.insert(d.end(), fsolve[J].begin(), fsolve[J].end());
        d.push_back(lastB[(size_t)J * nch + ch]);
        lastB[(size_t)J * nch + ch] = b.add_v(TASK_BGEMV, J, I, ch, c_gemv, d);
      }
  }
  return b.ordered(workers);
}

}  // namespace gpk
