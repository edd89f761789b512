/* Host-only use of the library from plain C99 through include/tn.h: circuit,
 * network and plan handles, plan determinism, the memory layout, error
 * reporting and NULL frees.
 * Prints one line "hash=<hex> slices=<n> steps=<n> bytes=<n>" on success and
 * exits non-zero on the first failed check. */
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

static int plan_bytes(const tn_network* net, uint8_t** bytes, size_t* len, tn_plan_info* info) {
  tn_plan_opts o;
  tn_plan_t* p = NULL;
  tn_tensor_layout* lay = NULL;
  int64_t arena[4], nt, x;
  memset(&o, 0, sizeof o);
  o.num_sliced = 2;
  o.search_trials = 8;
  o.seed = 3;
  CHECK(tn_plan(net, &o, &p) == TN_OK);
  CHECK(tn_plan_get_info(p, info) == TN_OK);
  CHECK(tn_plan_serialize(p, NULL, 0, len) == TN_OK && *len > 0);
  *bytes = (uint8_t*)malloc(*len);
  CHECK(*bytes != NULL);
  CHECK(tn_plan_serialize(p, *bytes, *len, len) == TN_OK);
  /* the layout: one entry per tensor, the root the only tensor nobody reads */
  nt = (int64_t)info->num_leaves + info->num_steps;
  lay = (tn_tensor_layout*)malloc((size_t)nt * sizeof *lay);
  CHECK(lay != NULL);
  CHECK(tn_plan_layout(p, lay, nt - 1, arena) == TN_EINVAL);
  CHECK(tn_plan_layout(p, lay, nt, arena) == TN_OK);
  for (x = 0; x < nt; ++x) {
    CHECK((lay[x].consumer < 0) == (x == nt - 1));
    CHECK(lay[x].offset >= 0 && lay[x].offset % 32 == 0);
  }
  CHECK(arena[0] > 0 && arena[2] > 0 && arena[3] > 0);
  free(lay);
  tn_free_plan(p);
  return 0;
}

int main(void) {
  tn_circuit* c = NULL;
  tn_network* net = NULL;
  int32_t n = 0;
  int64_t ng = 0;
  const int32_t open_q[2] = {14, 15};
  tn_network_info ni;
  tn_plan_info i1, i2;
  uint8_t *b1 = NULL, *b2 = NULL;
  size_t l1 = 0, l2 = 0;

  CHECK(strncmp(tn_version(), "gb300-rqc-tn", 12) == 0);
  /* errors: a status, a message, and the output left untouched */
  CHECK(tn_random_circuit(0, 4, 8, 1, &c) == TN_EINVAL && c == NULL);
  CHECK(strlen(tn_last_error()) > 0);
  CHECK(tn_build_network(NULL, NULL, 0, &net) == TN_EINVAL && net == NULL);

  CHECK(tn_random_circuit(4, 4, 8, 1, &c) == TN_OK);
  CHECK(tn_circuit_info(c, &n, &ng) == TN_OK && n == 16 && ng > 0);
  CHECK(tn_build_network(c, open_q, 2, &net) == TN_OK);
  CHECK(tn_network_get_info(net, &ni) == TN_OK && ni.num_open == 2 && ni.num_qubits == 16);
  CHECK(ni.num_closed == 14);

  /* equal inputs and seed give byte-identical plans */
  if (plan_bytes(net, &b1, &l1, &i1) || plan_bytes(net, &b2, &l2, &i2)) return 1;
  CHECK(l1 == l2 && memcmp(b1, b2, l1) == 0 && i1.hash == i2.hash);
  CHECK(i1.num_sliced == 2 && i1.num_slices == 4 && i1.num_open == 2);

  printf("hash=%llx slices=%lld steps=%d bytes=%zu\n", (unsigned long long)i1.hash, (long long)i1.num_slices,
         i1.num_steps, l1);
  free(b1);
  free(b2);
  tn_free_network(net);
  tn_free_circuit(c);
  tn_free_network(NULL);
  tn_free_circuit(NULL);
  tn_free_plan(NULL);
  return 0;
}
