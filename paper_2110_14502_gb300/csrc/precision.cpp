// tn_precision_analysis: per-step precision from a pre-analysis.
//
// Paper: Sec. "A Mixed-Precision Computation Method via Adaptive Precision
// Scaling" -- not every part of the contraction is equally sensitive to the
// half-precision format; a pre-analysis run on a few paths finds the
// sensitive parts (the paper locates them near the slicing positions) and
// keeps those in the accurate format while the rest runs in the fast one.
//
// Here the parts are the plan's pairwise steps that can run on the tensor
// cores (every step after the plan-invariant phase whose GEMM shape fits).
// On a probe -- the given bitstrings over the first `probe_slices` slices --
// the analysis contracts
//   * the complex64 reference,
//   * every candidate step in the fast precision and the rest accurate, one
//     candidate at a time: the error this step alone brings in,
// orders the candidates by that error and finds, by doubling and then
// bisection on the number of steps kept accurate (most sensitive first), the
// fewest accurate steps whose mixed assignment meets the target error on the
// probe.  Every contraction goes through the executor with a per-step
// precision array, so the analysis runs the same kernels as the hot path.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "kernels.h"
#include "tn_internal.h"

namespace tn {

namespace {

double rel_l2(const std::vector<double>& a, const std::vector<double>& ref) {
  double num = 0, den = 0;
  for (size_t i = 0; i < ref.size(); ++i) {
    num += (a[i] - ref[i]) * (a[i] - ref[i]);
    den += ref[i] * ref[i];
  }
  return den > 0 ? std::sqrt(num / den) : std::sqrt(num);
}

}  // namespace

}  // namespace tn

using namespace tn;

extern "C" tn_status tn_precision_analysis(tn_plan_t* p, const uint64_t* bitstrings, int64_t nb, int64_t probe_slices,
                                           int32_t fast_precision, int32_t accurate_precision, double target_rel_err,
                                           int8_t* step_precision, tn_precision_report* rep) {
  if (!p || !bitstrings || !step_precision) return fail(TN_EINVAL, "tn_precision_analysis: NULL argument");
  if (nb < 1 || nb > 4096) return fail(TN_EINVAL, "tn_precision_analysis: %lld probe bitstrings (1 .. 4096)", (long long)nb);
  auto tc_prec = [](int32_t x) { return x >= TN_PREC_SPLIT_BF16 && x <= TN_PREC_SCALED_BF16; };
  if (!tc_prec(fast_precision) || !tc_prec(accurate_precision))
    return fail(TN_EINVAL, "tn_precision_analysis: fast and accurate precisions must be 16-bit tensor-core ones");
  if (!(target_rel_err > 0)) return fail(TN_EINVAL, "tn_precision_analysis: target error must be > 0");
  const Plan& P = p->plan;
  const int64_t S_all = num_slice_ids(P);
  if (probe_slices < 1 || probe_slices > S_all)
    return fail(TN_EINVAL, "tn_precision_analysis: probe of %lld slices outside [1, 2^%zu]", (long long)probe_slices,
                P.sliced.size());
  return guarded("tn_precision_analysis", [&]() -> tn_status {
    const size_t ns = P.steps.size();
    const int k = (int)P.net.open_qubits.size();
    const int64_t nout = nb << k;
    // candidates: steps after phase 0 whose GEMM can run on the tensor cores
    std::vector<int> cand;
    for (size_t s = 0; s < ns; ++s) {
      if (P.steps[s].phase == 0 || P.steps[s].klass == SC_VECTOR) continue;
      GemmDesc d;
      make_gemm_desc(P.steps[s].la, P.steps[s].lb, P.steps[s].lc, d);
      if (tc_shape_ok(d) && !stream_preferred(d)) cand.push_back((int)s);
    }
    int runs = 0;
    auto contract = [&](int prec, const int8_t* sp, std::vector<double>& out) -> tn_status {
      tn_exec_opts o;
      std::memset(&o, 0, sizeof o);
      o.precision = prec;
      o.slice_begin = 0;
      o.slice_count = probe_slices;
      o.step_precision = sp;
      out.assign(2 * nout, 0.0);
      ++runs;
      return contract_amplitudes(p->plan, bitstrings, nb, out.data(), o, nullptr);
    };
    std::vector<double> ref, got;
    tn_status st = contract(TN_PREC_C64, nullptr, ref);
    if (st != TN_OK) return st;
    std::vector<int8_t> sp(ns, -1);
    auto assign = [&](const std::vector<int>& order, size_t accurate) {
      std::fill(sp.begin(), sp.end(), (int8_t)-1);
      for (size_t i = 0; i < order.size(); ++i) sp[order[i]] = (int8_t)(i < accurate ? accurate_precision : fast_precision);
    };
    auto err_of = [&](double& e) -> tn_status {
      tn_status r = contract(TN_PREC_C64, sp.data(), got);
      if (r == TN_OK) e = rel_l2(got, ref);
      return r;
    };
    // the error each candidate brings in alone (the others accurate)
    std::vector<double> sens(ns, 0.0);
    for (int s : cand) {
      for (int t : cand) sp[t] = (int8_t)accurate_precision;
      sp[s] = (int8_t)fast_precision;
      st = err_of(sens[s]);
      if (st != TN_OK) return st;
    }
    std::vector<int> order = cand;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return sens[a] > sens[b]; });
    double e_fast = 0, e_acc = 0;
    assign(order, 0);
    if ((st = err_of(e_fast)) != TN_OK) return st;
    assign(order, order.size());
    if ((st = err_of(e_acc)) != TN_OK) return st;
    // fewest accurate steps (most sensitive first) meeting the target
    size_t lo = 0, hi = order.size();  // err(lo) > target (unless lo = 0 passes), err(hi) is the best we have
    double e_best = e_acc;
    if (e_fast <= target_rel_err) {
      hi = 0;
      e_best = e_fast;
    } else {
      size_t m = 1;
      while (m < order.size()) {
        double e;
        assign(order, m);
        if ((st = err_of(e)) != TN_OK) return st;
        if (e <= target_rel_err) {
          hi = m;
          e_best = e;
          break;
        }
        lo = m;
        m *= 2;
      }
      while (hi - lo > 1) {
        const size_t mid = (lo + hi) / 2;
        double e;
        assign(order, mid);
        if ((st = err_of(e)) != TN_OK) return st;
        if (e <= target_rel_err) {
          hi = mid;
          e_best = e;
        } else {
          lo = mid;
        }
      }
    }
    assign(order, hi);
    std::memcpy(step_precision, sp.data(), ns);
    if (rep) {
      std::memset(rep, 0, sizeof *rep);
      rep->err_fast = e_fast;
      rep->err_accurate = e_acc;
      rep->err_mixed = e_best;
      rep->candidate_steps = (int32_t)cand.size();
      rep->accurate_steps = (int32_t)hi;
      double all = 0, acc = 0;
      int slice_dep = 0;
      for (size_t i = 0; i < order.size(); ++i) {
        const Step& S = P.steps[order[i]];
        // counted work of the step per slice (phase 1) or per slice and bitstring (phase 2)
        const double w = std::ldexp(1.0, S.nm + S.nn + S.nk) * (S.phase == 2 ? (double)nb : 1.0);
        all += w;
        if (i < hi) {
          acc += w;
          slice_dep += S.phase == 1;
        }
      }
      rep->accurate_flops_fraction = all > 0 ? acc / all : 0.0;
      rep->accurate_slice_only_steps = slice_dep;
      rep->probe_runs = runs;
    }
    return TN_OK;
  });
}
