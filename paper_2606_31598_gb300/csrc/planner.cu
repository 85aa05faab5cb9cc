// planner.cu -- the analytic memory-constrained planner of Sec. IV.B
// (Algorithm 1) as host code: workspace, operator memory, feasibility,
// arithmetic scale, task waves and the model score of one candidate plan.
// No GPU is touched here.
#include <algorithm>
#include <cmath>

#include "mf_internal.h"

namespace mf {

void planner_estimate(const mf_problem& pr, const mf_candidate& c, const mf_device_model& dm, double alpha,
                      double cache_budget, mf_estimate& e) {
  const double Dout = (double)pr.D_out, Din = (double)pr.D_in, R = (double)pr.R, nop = (double)pr.n_op;
  const double Bc = pr.B_c;
  const int64_t b = c.block > 0 ? c.block : pr.D_in;
  e.n_blk = (pr.D_in + b - 1) / b;
  e.n_pair = e.n_blk * (e.n_blk + 1) / 2;
  e.M_block = Bc * (double)b * (double)b;                                   // S_block = B_c b^2
  e.M_work = (double)c.r_arrays * Din * R * Bc;                             // Eq. planner_workspace
  const int32_t prow = std::max(1, c.p_row);
  const double m_full = nop * Dout * Din * Bc / (double)prow;              // Eq. planner_full_cache
  int64_t pc = c.pairs_cached;
  if (c.storage == MF_STORE_PARTIAL && pc < 0)                              // Eq. partial_cache_pairs
    pc = (int64_t)std::min<double>((double)e.n_pair, std::floor(cache_budget / e.M_block));
  if (c.storage == MF_STORE_FULL) pc = e.n_pair;
  if (c.storage == MF_STORE_PROCEDURAL) pc = 0;
  e.pairs_cached = pc;
  const double m_partial = nop * (double)pc * (double)b * (double)b * Bc;  // Eq. planner_partial_cache
  e.M_op = c.storage == MF_STORE_FULL ? m_full : (c.storage == MF_STORE_PARTIAL ? m_partial : 0.0);
  e.M_tot = e.M_op + e.M_work;                                              // Eq. planner_total_memory
  e.feasible = e.M_tot <= alpha * pr.M_free ? 1 : 0;                        // Eq. planner_memory_constraint
  e.F_mv = 8.0 * nop * Dout * Din * R;                                      // Eq. generic_matvec_flops
  const int64_t groups = std::max<int64_t>(1, c.groups);
  e.waves = (pr.N_task + groups - 1) / groups;                              // Eq. planner_waves
  // Runtime model (Sec. V.A, Eq. runtime_overlap): source access and the
  // contraction overlap, so one application costs the slowest of
  //   generation of the procedural canonical entries,
  //   streaming of the cached canonical entries,
  //   the contraction itself.
  const double canon = nop * Din * (Din + 1) / 2.0;
  const double frac_cached = e.n_pair > 0 ? (double)pc / (double)e.n_pair : 0.0;
  // the row-owner form (more than 16 vectors) generates each canonical
  // entry twice, the Hermitian forms once
  const double reuse = R > 16 ? 2.0 : 1.0;
  const double gen_entries = canon * (1.0 - frac_cached) * reuse;
  const double t_gen = dm.gen_entries_per_s > 0 ? gen_entries / dm.gen_entries_per_s : 0.0;
  const double t_mem = dm.hbm_bytes_per_s > 0 ? canon * frac_cached * Bc * reuse / dm.hbm_bytes_per_s : 0.0;
  const double t_mv = dm.flops_per_s > 0 ? e.F_mv / dm.flops_per_s : 0.0;
  e.T_model = std::max(t_gen, std::max(t_mem, t_mv));
  e.T_sum = t_gen + t_mem + t_mv;
  // Pi_mem: a 10 % penalty rising linearly over the last fifth of the
  // allowed memory (Eq. planner_cost_score leaves the form open).
  const double use = pr.M_free > 0 ? e.M_tot / (alpha * pr.M_free) : 0.0;
  const double pi_mem = 1.0 + 0.1 * std::max(0.0, std::min(1.0, (use - 0.8) / 0.2));
  e.S_model = (double)e.waves * e.T_model * pi_mem;                         // Eq. planner_cost_score
}

}  // namespace mf

extern "C" mf_status mf_planner_estimate(const mf_problem* prob, const mf_candidate* cand,
                                         const mf_device_model* model, double alpha, double cache_budget_bytes,
                                         mf_estimate* out) {
  if (!prob || !cand || !out || prob->D_in < 1 || prob->D_out < 1 || prob->R < 1 || prob->n_op < 1 ||
      prob->N_task < 1 || !(prob->B_c > 0) || !(alpha > 0 && alpha <= 1) || cand->block < 0 ||
      cand->storage < MF_STORE_PROCEDURAL || cand->storage > MF_STORE_FULL)
    return MF_ERR_INVALID;
  mf_device_model dm{};
  if (model) dm = *model;
  mf::planner_estimate(*prob, *cand, dm, alpha, cache_budget_bytes, *out);
  return MF_OK;
}
