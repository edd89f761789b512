/* The hot path from plain C99 through include/tn.h: a seeded circuit, its
 * network and a sliced plan, tn_contract_amplitudes with host buffers in two
 * precisions, and one request through the serving API.
 * argv[1..]: bitstrings as hexadecimal 64-bit words (qubit q = bit q).
 * Prints, per precision and per bitstring, one line
 *   "<tag> <b> <j> <re> <im>"
 * for every amplitude j of the batch (tags c64, split_fp16, served), and exits
 * non-zero on the first failed call. */
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "tn.h"

#define CHECK(cond)                                                           \
  do {                                                                        \
    if (!(cond)) {                                                            \
      fprintf(stderr, "check failed at line %d: %s (%s)\n", __LINE__, #cond, \
              tn_last_error());                                               \
      return 1;                                                               \
    }                                                                         \
  } while (0)

#define ROWS 4
#define COLS 5
#define DEPTH 12
#define SEED 15
#define NOPEN 3

int main(int argc, char** argv) {
  tn_circuit* c = NULL;
  tn_network* net = NULL;
  tn_plan_t* p = NULL;
  tn_plan_opts po;
  tn_exec_opts eo;
  tn_report rep;
  tn_server* srv = NULL;
  tn_server_opts so;
  tn_request rq;
  tn_request_stats st;
  int32_t open_q[NOPEN];
  uint64_t* bits;
  double* out;
  int64_t nb = argc - 1, ticket = 0, b, j, nout;
  int q, prec;
  const int precs[2] = {TN_PREC_C64, TN_PREC_SPLIT_FP16};
  const char* tags[2] = {"c64", "split_fp16"};

  CHECK(nb >= 1);
  bits = (uint64_t*)malloc((size_t)nb * sizeof *bits);
  nout = nb << NOPEN;
  out = (double*)malloc((size_t)nout * 2 * sizeof *out);
  CHECK(bits != NULL && out != NULL);
  for (b = 0; b < nb; ++b) bits[b] = strtoull(argv[b + 1], NULL, 16);
  for (q = 0; q < NOPEN; ++q) open_q[q] = ROWS * COLS - NOPEN + q;

  CHECK(tn_random_circuit(ROWS, COLS, DEPTH, SEED, &c) == TN_OK);
  CHECK(tn_build_network(c, open_q, NOPEN, &net) == TN_OK);
  memset(&po, 0, sizeof po);
  po.num_sliced = 4;
  po.search_trials = 16;
  po.seed = 1;
  CHECK(tn_plan(net, &po, &p) == TN_OK);

  for (prec = 0; prec < 2; ++prec) {
    memset(&eo, 0, sizeof eo);
    eo.precision = precs[prec];
    eo.slice_count = -1;  /* every slice */
    memset(out, 0, (size_t)nout * 2 * sizeof *out);
    CHECK(tn_contract_amplitudes(p, bits, nb, out, &eo, &rep) == TN_OK);
    CHECK(rep.units == nb * 16 && rep.kernel_launches > 0);
    for (b = 0; b < nb; ++b)
      for (j = 0; j < (1 << NOPEN); ++j)
        printf("%s %lld %lld %.17g %.17g\n", tags[prec], (long long)b, (long long)j,
               out[2 * ((b << NOPEN) + j)], out[2 * ((b << NOPEN) + j) + 1]);
  }

  /* one request through the continuous-batching server */
  memset(&so, 0, sizeof so);
  so.max_inflight = 2;
  so.slices_per_quantum = 4;
  so.precision = TN_PREC_C64;
  so.plan_trials = 8;
  so.max_log2_intermediate = 12;
  CHECK(tn_server_create(&so, &srv) == TN_OK);
  memset(&rq, 0, sizeof rq);
  rq.rows = ROWS;
  rq.cols = COLS;
  rq.depth = DEPTH;
  rq.num_open = NOPEN;
  rq.seed = SEED;
  rq.nb = nb;
  rq.bitstrings = bits;
  rq.precision = -1;
  CHECK(tn_submit(srv, &rq, &ticket) == TN_OK);
  memset(out, 0, (size_t)nout * 2 * sizeof *out);
  CHECK(tn_wait(srv, ticket, out, nout, &st, 0.0) == TN_OK);
  CHECK(st.status == TN_OK && st.nb == nb && st.quanta >= 1 && st.gpu_end_ms >= st.gpu_begin_ms);
  for (b = 0; b < nb; ++b)
    for (j = 0; j < (1 << NOPEN); ++j)
      printf("served %lld %lld %.17g %.17g\n", (long long)b, (long long)j, out[2 * ((b << NOPEN) + j)],
             out[2 * ((b << NOPEN) + j) + 1]);
  tn_server_destroy(srv);

  tn_free_plan(p);
  tn_free_network(net);
  tn_free_circuit(c);
  free(bits);
  free(out);
  return 0;
}
