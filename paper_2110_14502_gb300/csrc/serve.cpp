// Serving: continuous batching of amplitude requests on one GPU.
//
// The paper's parallelisation (Sec. "A Customized Parallelization Scheme")
// treats slices as independent sub-tasks; here the same independence lets one
// GPU interleave the slices of many requests.  Requests for circuits of any
// grid size and depth arrive at any time (tn_submit, any thread).  A planner
// thread builds each request's network and plan (plans are cached per circuit
// and open-qubit count; every admitted request gets its own copy with its own
// device state, so a copy never shares buffers).  A scheduler thread admits
// planned requests in arrival order while an in-flight slot is free and their
// estimated device footprint fits the HBM budget, then interleaves them: each
// turn queues one quantum (a group of consecutive slices) of every admitted
// request on that request's own CUDA stream, so the requests' work overlaps on
// the device.  A request whose slices are all queued gets its amplitudes copied
// back; when that copy has completed it is done, its slot and budget are freed
// and the next requests are admitted.  Requests for the same circuit, open
// qubits, precision and slice range that wait for admission together are
// served as one contraction: their bitstrings become units of the same
// launches, and each gets its own rows of the result.  The FP64 sum of a request runs in slice
// order whatever else is in flight, so a result is bit-identical alone and in
// the mix.  Requests whose plan exceeds the cost cap fail with TN_ETOOBIG, and
// ones that could never fit the budget with TN_EHBM; neither is dropped silently.
#include <algorithm>
#include <cmath>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <tuple>
#include <vector>

#include <cuda_runtime.h>

#include "tn_internal.h"

namespace tn {

namespace {

using Clock = std::chrono::steady_clock;

enum ReqState { RS_PENDING, RS_READY, RS_ACTIVE, RS_FINISHING, RS_DONE };

struct PlanKey {
  int rows, cols, depth, open;
  uint64_t seed;
  int trials, width;
  double cap;
  bool operator<(const PlanKey& o) const {
    return std::tie(rows, cols, depth, open, seed, trials, width, cap) <
           std::tie(o.rows, o.cols, o.depth, o.open, o.seed, o.trials, o.width, o.cap);
  }
};

struct Request {
  int64_t ticket = 0;
  tn_request params{};
  std::vector<uint64_t> bits;
  int32_t precision = 0;
  ReqState state = RS_PENDING;
  tn_status status = TN_OK;
  std::string error;
  std::unique_ptr<tn_plan_s> plan;  // own copy: own device state
  int64_t ns = 0, cursor = 0, q = 1;
  int64_t footprint = 0;
  int words = 1, k = 0;
  uint64_t* d_bits = nullptr;
  double* d_acc = nullptr;
  double* h_out = nullptr;  // pinned
  cudaStream_t stream = nullptr;
  cudaEvent_t done_ev = nullptr;
  std::vector<cudaEvent_t> quanta;  // events of queued quanta (bounded look-ahead)
  // device timeline: timing events before the first quantum and after the
  // last one, read against the server's epoch once the request is done
  cudaEvent_t ev_begin = nullptr, ev_end = nullptr;
  int64_t nquanta = 0;
  double gpu_begin_ms = 0, gpu_end_ms = 0;
  Clock::time_point t_submit, t_admit, t_done;
  bool planned_here = false;
  PlanKey key{};
  int64_t nb_own = 0;  // this request's bitstrings (the first rows of the contraction it leads)
  // requests served in this one's contraction (their bitstrings follow its own)
  std::vector<std::shared_ptr<Request>> members;
  int64_t batched = 1;  // requests in the contraction that served this one
  bool member = false;  // served in another request's contraction
  int stem_reused = 0;  // whether the contraction that served it reused a resident stem (set when done)
};



// Plans are pure functions of the circuit and the planning options, so one
// cache serves every server of the process (host memory only: copies of a
// cached plan own their device state).  It holds the kPlanCacheSize most
// recently used plans.
constexpr size_t kPlanCacheSize = 256;
// bitstrings of requests merged into one contraction (one launch group)
constexpr int64_t kMergeBits = 256;
struct CachedPlan {
  std::shared_ptr<tn_plan_s> plan;
  uint64_t last = 0;
};
std::mutex g_plan_mu;
std::map<PlanKey, CachedPlan> g_plan_cache;
uint64_t g_plan_clock = 0;

}  // namespace

struct Server {
  tn_server_opts opts{};
  int device = 0;
  std::mutex mu;
  std::condition_variable cv;
  bool stop = false;
  int64_t next_ticket = 1;
  std::map<int64_t, std::shared_ptr<Request>> reqs;
  std::deque<std::shared_ptr<Request>> to_plan, ready;
  std::vector<std::shared_ptr<Request>> active;
  // done requests whose executors (device memory) still count against the
  // budget until the client waits for them or admission needs the room
  std::deque<std::shared_ptr<Request>> held;
  int64_t budget = 0, in_use = 0;
  // stems (leaf store + phase-0 outputs) of recent circuits, resident for
  // later requests of the same circuit; its capacity is taken off the budget
  std::shared_ptr<StemCache> stems;
  std::vector<cudaStream_t> streams;  // one per slot
  cudaEvent_t epoch = nullptr;        // device time zero of the request timelines
  std::vector<std::thread> planners;
  std::thread scheduler;
};

namespace {

// Device memory of a request (nb = params.nb bitstrings) running quanta of q
// slices: arenas (8 bytes per complex64 element) and the operand planes of a
// split pass (at most 8 bytes per element of the step's two operands, which
// the arena holds side by side) of one quantum, leaves, invariants, I/O.
int64_t footprint(const Request& R, int64_t q) {
  const Plan& P = R.plan->plan;
  const int64_t gb = std::min<int64_t>(std::max<int64_t>(R.params.nb, 1), 256);
  return 16 * q * (P.slice_arena_elems + gb * P.unit_arena_elems) + 8 * (P.invariant_elems + P.leaf_store_elems) +
         16 * (R.params.nb << R.k) + (int64_t(32) << 20);
}

tn_status plan_request(Server& S, Request& R) {
  const tn_request& p = R.params;
  // the cost cap bounds the work served: a request of fidelity f runs a
  // fraction f of the slices, so its plan may cost up to 2^cap / f in full
  const double f = p.fidelity;
  const bool partial = f > 0.0 && f < 1.0;
  // over_cap_policy 1: plan without a cost cap and serve the slices that fit
  const bool fit = S.opts.over_cap_policy == 1 && !partial;
  const double cap = fit ? 1000.0 : S.opts.max_log2_cmac + (partial ? -std::log2(f) : 0.0);
  PlanKey key{p.rows, p.cols, p.depth, p.num_open, p.seed, S.opts.plan_trials, S.opts.max_log2_intermediate, cap};
  R.key = key;
  std::shared_ptr<tn_plan_s> cached;
  {
    std::lock_guard<std::mutex> g(g_plan_mu);
    auto it = g_plan_cache.find(key);
    if (it != g_plan_cache.end()) {
      cached = it->second.plan;
      it->second.last = ++g_plan_clock;
    }
  }
  if (!cached) {
    tn_circuit* c = nullptr;
    tn_status st = tn_random_circuit(p.rows, p.cols, p.depth, p.seed, &c);
    if (st != TN_OK) return st;
    const int n = p.rows * p.cols;
    std::vector<int32_t> open;
    for (int q = n - p.num_open; q < n; ++q) open.push_back(q);
    tn_network* net = nullptr;
    st = tn_build_network(c, open.data(), (int32_t)open.size(), &net);
    tn_free_circuit(c);
    if (st != TN_OK) return st;
    tn_plan_opts po{};
    po.num_sliced = -1;
    po.max_log2_intermediate = S.opts.max_log2_intermediate;
    po.search_trials = S.opts.plan_trials;
    po.seed = 1;
    po.max_log2_cmac = cap;
    tn_plan_t* pl = nullptr;
    st = tn_plan(net, &po, &pl);
    tn_free_network(net);
    if (st != TN_OK) return st;
    cached.reset(pl);
    R.planned_here = true;
    std::lock_guard<std::mutex> g(g_plan_mu);
    if (g_plan_cache.size() >= kPlanCacheSize && !g_plan_cache.count(key)) {
      auto oldest = g_plan_cache.begin();
      for (auto i = g_plan_cache.begin(); i != g_plan_cache.end(); ++i)
        if (i->second.last < oldest->second.last) oldest = i;
      g_plan_cache.erase(oldest);  // requests still holding it keep their own copy
    }
    g_plan_cache[key] = CachedPlan{cached, ++g_plan_clock};
  }
  auto* copy = new (std::nothrow) tn_plan_s(cached->plan);
  if (!copy) return fail(TN_ENOMEM, "serving: out of host memory");
  copy->plan.stems = S.stems;
  R.plan.reset(copy);
  const Plan& P = R.plan->plan;
  // fidelity by fraction: the first ceil(f 2^S) slices (all for f = 0 or 1)
  const int64_t all = num_slice_ids(P);
  R.ns = partial ? std::max<int64_t>(1, std::min<int64_t>(all, (int64_t)std::ceil(f * (double)all))) : all;
  if (fit) {
    // the largest leading range of slices whose work fits the cap
    const double full = std::log2(std::max(1.0, P.cmac_per_slice)) + (double)P.sliced.size();
    if (full > S.opts.max_log2_cmac) {
      const double fits = std::floor(std::exp2(S.opts.max_log2_cmac) / std::max(1.0, P.cmac_per_slice));
      if (fits < 1.0)
        return fail(TN_ETOOBIG, "serving: one slice costs 2^%.1f CMAC, above the cap 2^%.1f",
                    std::log2(P.cmac_per_slice), S.opts.max_log2_cmac);
      R.ns = std::min<int64_t>(all, (int64_t)std::min(fits, 4.0e18));
    }
  }
  // rounding up to whole slices can serve more than f of the work
  const double served = std::log2(std::max(1.0, (double)R.ns * P.cmac_per_slice));
  if (partial && served > S.opts.max_log2_cmac)
    return fail(TN_ETOOBIG, "serving: %lld of %lld slices cost 2^%.1f CMAC, above the cap 2^%.1f", (long long)R.ns,
                (long long)all, served, S.opts.max_log2_cmac);
  R.q = std::min<int64_t>(R.ns, std::max(1, S.opts.slices_per_quantum));
  R.k = (int)P.net.open_qubits.size();
  R.words = std::max(1, (P.net.n + 63) / 64);
  // a request whose quantum would not fit in a quarter of the budget runs
  // smaller quanta (down to one slice), so that several requests still fit
  // side by side
  const int64_t per_slice = footprint(R, 1) - footprint(R, 0);
  const int64_t share = S.budget / 4 - footprint(R, 0);
  if (share > per_slice) R.q = std::min<int64_t>(R.q, share / per_slice);
  else R.q = 1;
  R.footprint = footprint(R, R.q);
  return TN_OK;
}

void planner_loop(Server* S) {
  cudaSetDevice(S->device);
  for (;;) {
    std::shared_ptr<Request> R;
    {
      std::unique_lock<std::mutex> g(S->mu);
      S->cv.wait(g, [&] { return S->stop || !S->to_plan.empty(); });
      if (S->stop) return;
      R = S->to_plan.front();
      S->to_plan.pop_front();
    }
    tn_status st = guarded("serving: planning", [&] { return plan_request(*S, *R); });
    std::lock_guard<std::mutex> g(S->mu);
    if (st != TN_OK) {
      R->status = st;
      R->error = tn_last_error();
      R->state = RS_DONE;
      R->t_done = Clock::now();
    } else if (R->footprint > S->budget) {
      R->status = fail(TN_EHBM, "serving: request %lld needs about %lld bytes, the budget is %lld",
                       (long long)R->ticket, (long long)R->footprint, (long long)S->budget);
      R->error = tn_last_error();
      R->state = RS_DONE;
      R->t_done = Clock::now();
    } else {
      R->state = RS_READY;
      S->ready.push_back(R);
    }
    S->cv.notify_all();
  }
}

// A done request gives back its stream-ordered buffers and events and waits
// in S.held for its executor to be freed.  Called with the server's mutex held.
void release(Server& S, const std::shared_ptr<Request>& Rp) {
  Request& R = *Rp;
  cudaFreeAsync(R.d_bits, R.stream);
  cudaFreeAsync(R.d_acc, R.stream);
  R.d_bits = nullptr;
  R.d_acc = nullptr;
  for (auto ev : R.quanta) cudaEventDestroy(ev);
  R.quanta.clear();
  if (R.done_ev) cudaEventDestroy(R.done_ev);
  R.done_ev = nullptr;
  if (R.ev_begin) cudaEventDestroy(R.ev_begin);
  if (R.ev_end) cudaEventDestroy(R.ev_end);
  R.ev_begin = R.ev_end = nullptr;
  R.stem_reused = R.plan && stem_reused(R.plan->plan) ? 1 : 0;
  // The plan copy's executor (arenas, operand planes, graphs) keeps its device
  // memory, and its budget share, until the client waits for the request or
  // admission needs the room (reclaim); freeing device memory synchronises the
  // device, so it is not done on every completion.
  S.held.push_back(Rp);
}

// Frees the executors of held requests, oldest first, until `need` more
// bytes fit the budget (or none is left).  Called with the server's mutex held.
void reclaim(Server& S, int64_t need) {
  while (!S.held.empty() && S.in_use + need > S.budget) {
    std::shared_ptr<Request> R = S.held.front();
    S.held.pop_front();
    if (R->plan && R->plan->plan.exec) {
      destroy_executor(R->plan->plan.exec);
      R->plan->plan.exec = nullptr;
    }
    S.in_use -= R->footprint;
  }
}

tn_status admit(Server&, Request& R, cudaStream_t stream) {
  R.stream = stream;
  const int64_t nout = R.params.nb << R.k;
  cudaError_t e = cudaMallocAsync(&R.d_bits, std::max<int64_t>(R.bits.size(), 1) * sizeof(uint64_t), stream);
  if (e == cudaSuccess) e = cudaMallocAsync(&R.d_acc, std::max<int64_t>(nout, 1) * 16, stream);
  if (e == cudaSuccess && !R.bits.empty())
    e = cudaMemcpyAsync(R.d_bits, R.bits.data(), R.bits.size() * sizeof(uint64_t), cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess && !R.h_out) e = cudaMallocHost(&R.h_out, std::max<int64_t>(nout, 1) * 16);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&R.done_ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreate(&R.ev_begin);
  if (e == cudaSuccess) e = cudaEventCreate(&R.ev_end);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(TN_ECUDA, "serving: admitting request %lld: %s", (long long)R.ticket, cudaGetErrorString(e));
  }
  R.t_admit = Clock::now();
  return TN_OK;
}

// Queue the next quantum of R (slices cursor .. cursor+q-1); at the end queue
// the copy of the amplitudes back.
tn_status step_request(Request& R) {
  tn_exec_opts o{};
  o.stream = R.stream;
  o.precision = R.precision;
  o.device_io = 1;
  o.slice_begin = R.cursor;
  o.slice_count = std::min<int64_t>(R.q, R.ns - R.cursor);
  o.units_per_group = (int32_t)R.q;
  o.use_graph = 1;
  // one FP64 sum over all quanta: the filter list is reset by the first
  // quantum and processed (recompute / discard) after the last
  const bool first = R.cursor == 0, last = R.cursor + o.slice_count >= R.ns;
  if (first && cudaEventRecord(R.ev_begin, R.stream) != cudaSuccess)
    return fail(TN_ECUDA, "serving: recording the request's first-quantum event");
  tn_status st = contract_amplitudes_ex(R.plan->plan, R.d_bits, R.params.nb, R.d_acc, o, nullptr, first,
                                        (first ? 1 : 0) | (last ? 2 : 0));
  if (st != TN_OK) return st;
  R.cursor += o.slice_count;
  ++R.nquanta;
  cudaEvent_t ev;
  if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess) {
    cudaEventRecord(ev, R.stream);
    R.quanta.push_back(ev);
  }
  if (R.cursor >= R.ns) {
    const int64_t nout = R.params.nb << R.k;
    cudaError_t e = cudaEventRecord(R.ev_end, R.stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(R.h_out, R.d_acc, std::max<int64_t>(nout, 1) * 16, cudaMemcpyDeviceToHost, R.stream);
    if (e == cudaSuccess) e = cudaEventRecord(R.done_ev, R.stream);
    if (e != cudaSuccess) return fail(TN_ECUDA, "serving: %s", cudaGetErrorString(e));
    R.state = RS_FINISHING;
  }
  return TN_OK;
}

// A contraction that served several requests is done: each member gets its
// rows of the result (after the leader's own), the leader's timings and
// status.  Called with the server's mutex held.
void finish_members(Request& R) {
  int64_t row = R.nb_own;
  const int64_t per = int64_t(1) << R.k;
  R.batched = 1 + (int64_t)R.members.size();
  for (auto& X : R.members) {
    X->status = R.status;
    X->error = R.error;
    X->t_admit = R.t_admit;
    X->t_done = R.t_done;
    X->gpu_begin_ms = R.gpu_begin_ms;
    X->gpu_end_ms = R.gpu_end_ms;
    X->nquanta = R.nquanta;
    X->k = R.k;
    X->batched = R.batched;
    X->member = true;
    X->stem_reused = R.plan && stem_reused(R.plan->plan) ? 1 : 0;
    if (R.status == TN_OK && R.h_out) {
      const int64_t n = X->nb_own * per;
      if (cudaMallocHost(&X->h_out, std::max<int64_t>(n, 1) * 16) == cudaSuccess) {
        std::memcpy(X->h_out, R.h_out + 2 * row * per, n * 16);
      } else {
        X->h_out = nullptr;
        X->status = TN_ENOMEM;
        X->error = "serving: pinned host memory for a merged request's result";
      }
    }
    row += X->nb_own;
    X->state = RS_DONE;
  }
  R.members.clear();
}

void scheduler_loop(Server* S) {
  cudaSetDevice(S->device);
  std::vector<char> slot_busy(S->streams.size(), 0);
  std::map<Request*, int> slot_of;
  for (;;) {
    std::vector<std::shared_ptr<Request>> act;
    {
      std::unique_lock<std::mutex> g(S->mu);
      if (S->stop) return;
      // admission: arrival order, a free slot and room in the budget
      while (!S->ready.empty()) {
        // a copy: erasing merged requests from the deque below invalidates
        // references into it
        const std::shared_ptr<Request> R = S->ready.front();
        int slot = -1;
        for (size_t i = 0; i < slot_busy.size(); ++i)
          if (!slot_busy[i]) { slot = (int)i; break; }
        if (slot >= 0 && S->in_use + R->footprint > S->budget) reclaim(*S, R->footprint);
        if (slot < 0 || S->in_use + R->footprint > S->budget) break;
        // requests of the same circuit, precision and slices waiting behind
        // this one join its contraction while its bitstrings fit one group
        for (auto it = S->ready.begin() + 1; it != S->ready.end();) {
          Request& X = **it;
          const bool same = X.key.rows == R->key.rows && X.key.cols == R->key.cols && X.key.depth == R->key.depth &&
                            X.key.open == R->key.open && X.key.seed == R->key.seed && X.key.trials == R->key.trials &&
                            X.key.width == R->key.width && X.key.cap == R->key.cap && X.precision == R->precision &&
                            X.ns == R->ns;
          if (!same || R->params.nb + X.params.nb > kMergeBits) { ++it; continue; }
          R->params.nb += X.params.nb;
          const int64_t fp = footprint(*R, R->q);
          if (S->in_use + fp > S->budget) reclaim(*S, fp);
          if (S->in_use + fp > S->budget) {
            R->params.nb -= X.params.nb;
            ++it;
            continue;
          }
          R->footprint = fp;
          R->bits.insert(R->bits.end(), X.bits.begin(), X.bits.end());
          X.state = RS_ACTIVE;
          R->members.push_back(*it);
          it = S->ready.erase(it);
        }
        tn_status st = guarded("serving: admission", [&] { return admit(*S, *R, S->streams[slot]); });
        if (st != TN_OK) {
          R->status = st;
          R->error = tn_last_error();
          R->state = RS_DONE;
          R->t_done = Clock::now();
          finish_members(*R);
          S->ready.pop_front();
          S->cv.notify_all();
          continue;
        }
        slot_busy[slot] = 1;
        slot_of[R.get()] = slot;
        S->in_use += R->footprint;
        R->state = RS_ACTIVE;
        S->active.push_back(R);
        S->ready.pop_front();
      }
      act = S->active;
      if (act.empty()) {
        S->cv.wait_for(g, std::chrono::milliseconds(2));
        continue;
      }
    }
    bool progressed = false;
    for (auto& R : act) {
      if (R->state == RS_ACTIVE) {
        // bounded look-ahead: at most two quanta of a request in flight
        while (!R->quanta.empty() && cudaEventQuery(R->quanta.front()) == cudaSuccess) {
          cudaEventDestroy(R->quanta.front());
          R->quanta.erase(R->quanta.begin());
        }
        if (R->quanta.size() < 2) {
          tn_status st = guarded("serving: contraction", [&] { return step_request(*R); });
          progressed = true;
          if (st != TN_OK) {
            std::lock_guard<std::mutex> g(S->mu);
            cudaStreamSynchronize(R->stream);
            R->status = st;
            R->error = tn_last_error();
            R->state = RS_DONE;
            R->t_done = Clock::now();
            finish_members(*R);
            release(*S, R);
            slot_busy[slot_of[R.get()]] = 0;
            slot_of.erase(R.get());
            S->active.erase(std::find(S->active.begin(), S->active.end(), R));
            S->cv.notify_all();
          }
        }
      } else if (R->state == RS_FINISHING && cudaEventQuery(R->done_ev) == cudaSuccess) {
        std::lock_guard<std::mutex> g(S->mu);
        float b = 0.f, e = 0.f;
        if (cudaEventElapsedTime(&b, S->epoch, R->ev_begin) == cudaSuccess &&
            cudaEventElapsedTime(&e, S->epoch, R->ev_end) == cudaSuccess) {
          R->gpu_begin_ms = b;
          R->gpu_end_ms = e;
        }
        R->t_done = Clock::now();
        R->state = RS_DONE;
        finish_members(*R);
        release(*S, R);
        slot_busy[slot_of[R.get()]] = 0;
        slot_of.erase(R.get());
        S->active.erase(std::find(S->active.begin(), S->active.end(), R));
        progressed = true;
        S->cv.notify_all();
      }
    }
    if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(200));
  }
}

}  // namespace

}  // namespace tn

using namespace tn;

struct tn_server_s {
  Server s;
};

extern "C" tn_status tn_server_create(const tn_server_opts* opts, tn_server** out) {
  if (!out) return fail(TN_EINVAL, "tn_server_create: out is NULL");
  auto* h = new (std::nothrow) tn_server_s;
  if (!h) return fail(TN_ENOMEM, "tn_server_create: out of host memory");
  Server& S = h->s;
  if (opts) S.opts = *opts;
  if (S.opts.max_inflight <= 0) S.opts.max_inflight = 4;
  if (S.opts.max_inflight > 64) S.opts.max_inflight = 64;
  if (S.opts.slices_per_quantum <= 0) S.opts.slices_per_quantum = 64;
  if (S.opts.plan_trials <= 0) S.opts.plan_trials = 16;
  if (S.opts.max_log2_cmac <= 0) S.opts.max_log2_cmac = 48.0;
  if (S.opts.max_log2_intermediate <= 0) S.opts.max_log2_intermediate = 27;
  if (S.opts.precision < TN_PREC_C64 || S.opts.precision > TN_PREC_SCALED_BF16) {
    const int prec = S.opts.precision;  // S lives in h
    delete h;
    return fail(TN_EINVAL, "tn_server_create: unknown precision %d", prec);
  }
  if (cudaGetDevice(&S.device) != cudaSuccess) {
    delete h;
    return fail(TN_ENODEVICE, "tn_server_create: no CUDA device");
  }
  size_t freeb = 0, totb = 0;
  if (cudaMemGetInfo(&freeb, &totb) != cudaSuccess) {
    delete h;
    return fail(TN_ECUDA, "tn_server_create: cudaMemGetInfo failed");
  }
  const int64_t total = S.opts.hbm_budget_bytes > 0 ? S.opts.hbm_budget_bytes : (int64_t)(0.6 * (double)freeb);
  S.budget = total - total / 8;
  for (int i = 0; i < S.opts.max_inflight; ++i) {
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      for (auto x : S.streams) cudaStreamDestroy(x);
      delete h;
      return fail(TN_ECUDA, "tn_server_create: stream creation failed");
    }
    S.streams.push_back(st);
  }
  if (cudaEventCreate(&S.epoch) != cudaSuccess || cudaEventRecord(S.epoch, S.streams[0]) != cudaSuccess ||
      cudaEventSynchronize(S.epoch) != cudaSuccess) {
    if (S.epoch) cudaEventDestroy(S.epoch);
    for (auto x : S.streams) cudaStreamDestroy(x);
    delete h;
    return fail(TN_ECUDA, "tn_server_create: epoch event");
  }
  const int np_ = S.opts.planner_threads > 0 ? std::min(S.opts.planner_threads, 32) : 4;  // planner threads
  const tn_status st = guarded("tn_server_create", [&]() -> tn_status {
    S.stems = make_stem_cache(total / 8);
    for (int i = 0; i < np_; ++i) S.planners.push_back(std::thread(planner_loop, &S));
    S.scheduler = std::thread(scheduler_loop, &S);
    return TN_OK;
  });
  if (st != TN_OK) {
    const std::string msg = tn_last_error();
    tn_server_destroy(h);  // stops and joins the threads that did start
    return fail(st, "%s", msg.c_str());
  }
  *out = h;
  return TN_OK;
}

extern "C" tn_status tn_submit(tn_server* h, const tn_request* req, int64_t* ticket) {
  if (!h || !req || !ticket) return fail(TN_EINVAL, "tn_submit: NULL argument");
  const int n = req->rows >= 1 && req->rows <= 64 && req->cols >= 1 && req->cols <= 64 ? req->rows * req->cols : 0;
  if (n < 1 || n > 64 || req->depth < 0 || req->num_open < 0 || req->num_open > 12 ||
      req->num_open > n || req->nb < 1 || req->nb > (int64_t(1) << 24) || !req->bitstrings ||
      !(req->fidelity >= 0.0 && req->fidelity <= 1.0))
    return fail(TN_EINVAL, "tn_submit: bad request (grid %dx%d, depth %d, %d open, %lld bitstrings)", req->rows,
                req->cols, req->depth, req->num_open, (long long)req->nb);
  Server& S = h->s;
  const int32_t prec = req->precision < 0 ? S.opts.precision : req->precision;
  if (prec < TN_PREC_C64 || prec > TN_PREC_SCALED_BF16) return fail(TN_EINVAL, "tn_submit: unknown precision %d", prec);
  return guarded("tn_submit", [&]() -> tn_status {
  auto R = std::make_shared<Request>();
  R->params = *req;
  R->nb_own = req->nb;
  R->precision = prec;
  const int words = std::max(1, (n + 63) / 64);
  R->bits.assign(req->bitstrings, req->bitstrings + req->nb * words);
  R->params.bitstrings = nullptr;
  R->t_submit = Clock::now();
  std::lock_guard<std::mutex> g(S.mu);
  R->ticket = S.next_ticket++;
  S.reqs[R->ticket] = R;
  S.to_plan.push_back(R);
  S.cv.notify_all();
  *ticket = R->ticket;
  return TN_OK;
  });
}

extern "C" tn_status tn_poll(tn_server* h, int64_t ticket, int32_t* done) {
  if (!h || !done) return fail(TN_EINVAL, "tn_poll: NULL argument");
  std::lock_guard<std::mutex> g(h->s.mu);
  auto it = h->s.reqs.find(ticket);
  if (it == h->s.reqs.end()) return fail(TN_EINVAL, "tn_poll: unknown ticket %lld", (long long)ticket);
  *done = it->second->state == RS_DONE;
  return TN_OK;
}

extern "C" tn_status tn_wait(tn_server* h, int64_t ticket, double* out, int64_t capacity, tn_request_stats* stats,
                             double timeout_s) {
  if (!h) return fail(TN_EINVAL, "tn_wait: NULL server");
  Server& S = h->s;
  std::shared_ptr<Request> R;
  bool charged = false;
  {
    std::unique_lock<std::mutex> g(S.mu);
    auto it = S.reqs.find(ticket);
    if (it == S.reqs.end()) return fail(TN_EINVAL, "tn_wait: unknown ticket %lld", (long long)ticket);
    R = it->second;
    auto pred = [&] { return R->state == RS_DONE; };
    if (timeout_s > 0) {
      if (!S.cv.wait_for(g, std::chrono::duration<double>(timeout_s), pred))
        return fail(TN_ETIMEOUT, "tn_wait: request %lld not done after %.3f s", (long long)ticket, timeout_s);
    } else {
      S.cv.wait(g, pred);
    }
    S.reqs.erase(ticket);
    auto hit = std::find(S.held.begin(), S.held.end(), R);
    charged = hit != S.held.end();
    if (charged) S.held.erase(hit);
  }
  if (charged) {
    // the executor's device memory, then its budget share
    if (R->plan && R->plan->plan.exec) {
      destroy_executor(R->plan->plan.exec);
      R->plan->plan.exec = nullptr;
    }
    std::lock_guard<std::mutex> g(S.mu);
    S.in_use -= R->footprint;
    S.cv.notify_all();
  }
  const int64_t nout = R->nb_own << R->k;
  if (stats) {
    std::memset(stats, 0, sizeof *stats);
    auto ms = [](Clock::time_point a, Clock::time_point b) {
      return std::chrono::duration<double, std::milli>(b - a).count();
    };
    stats->submit_to_done_ms = ms(R->t_submit, R->t_done);
    stats->queue_ms = R->status == TN_OK ? ms(R->t_submit, R->t_admit) : 0.0;
    stats->device_ms = R->status == TN_OK ? ms(R->t_admit, R->t_done) : 0.0;
    stats->slices = R->ns;
    if (R->plan) stats->slice_fraction = (double)R->ns / std::ldexp(1.0, (int)R->plan->plan.sliced.size());
    stats->status = R->status;
    stats->num_open = R->k;
    stats->nb = R->nb_own;
    stats->batched_requests = R->batched;
    if (R->plan) {
      const Plan& P = R->plan->plan;
      // the slice-only work of a merged contraction is counted with its leader
      stats->flops = 8.0 * ((R->member ? 0.0 : (double)R->ns * P.cmac_slice_only) +
                            (double)R->nb_own * R->ns * (P.cmac_per_slice - P.cmac_slice_only));
      stats->plan_hash = P.hash;
    }
    stats->planned_here = R->planned_here;
    stats->stem_reused = R->stem_reused;
    stats->gpu_begin_ms = R->gpu_begin_ms;
    stats->gpu_end_ms = R->gpu_end_ms;
    stats->quanta = R->nquanta;
  }
  tn_status st = R->status;
  if (st == TN_OK && out) {
    if (capacity < nout) {
      st = fail(TN_EINVAL, "tn_wait: capacity %lld < %lld complex results", (long long)capacity, (long long)nout);
    } else {
      std::memcpy(out, R->h_out, nout * 16);
    }
  } else if (st != TN_OK) {
    fail(st, "%s", R->error.c_str());
  }
  if (R->h_out) cudaFreeHost(R->h_out);
  R->h_out = nullptr;
  R->plan.reset();
  return st;
}

extern "C" void tn_server_destroy(tn_server* h) {
  if (!h) return;
  Server& S = h->s;
  {
    std::lock_guard<std::mutex> g(S.mu);
    S.stop = true;
    S.cv.notify_all();
  }
  for (auto& t : S.planners)
    if (t.joinable()) t.join();
  if (S.scheduler.joinable()) S.scheduler.join();
  cudaDeviceSynchronize();
  for (auto& kv : S.reqs) {
    Request& R = *kv.second;
    if (R.d_bits) cudaFree(R.d_bits);
    if (R.d_acc) cudaFree(R.d_acc);
    if (R.h_out) cudaFreeHost(R.h_out);
    for (auto ev : R.quanta) cudaEventDestroy(ev);
    if (R.done_ev) cudaEventDestroy(R.done_ev);
    if (R.ev_begin) cudaEventDestroy(R.ev_begin);
    if (R.ev_end) cudaEventDestroy(R.ev_end);
    R.plan.reset();
  }
  if (S.epoch) cudaEventDestroy(S.epoch);
  for (auto x : S.streams) cudaStreamDestroy(x);
  delete h;
}
