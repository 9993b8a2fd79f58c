/* A C99 client of the C ABI using only its host entry points (no GPU needed): build a plan, read its
 * info and schedule description, parse and export OpenQASM, and check an error path. Compiled and
 * run by tests/test_c_client.py. */
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "qsim.h"

_Static_assert(sizeof(qsim_gate) == 24, "qsim_gate layout");
_Static_assert(sizeof(qsim_plan_opts) == 80, "qsim_plan_opts layout");
_Static_assert(sizeof(qsim_plan_info) == 48, "qsim_plan_info layout");

int main(void) {
  /* H(0), CNOT(0 -> 1), RY(theta_0) on 1, RX(input column 0) on 0 */
  qsim_gate g[4] = {{QSIM_H, {0, -1}, {-1, -1}, -1},
                    {QSIM_CNOT, {1, -1}, {0, -1}, -1},
                    {QSIM_RY, {1, -1}, {-1, -1}, 0},
                    {QSIM_RX, {0, -1}, {-1, -1}, -2}};
  qsim_plan_opts o;
  qsim_default_opts(&o);
  qsim_plan_t p = NULL;
  int rc = qsim_plan(g, 4, 2, &o, &p);
  if (rc != QSIM_OK || p == NULL) {
    printf("plan failed: %d %s\n", rc, qsim_last_error());
    return 1;
  }
  qsim_plan_info info;
  if (qsim_plan_info_get(p, &info) != QSIM_OK) return 2;
  printf("info %d %d %d %d %d\n", info.n_qubits, info.n_gates, info.n_params, info.n_inputs, info.n_passes);
  size_t need = 0;
  if (qsim_plan_describe(p, NULL, 0, &need) != QSIM_OK || need < 2) return 3;
  char* buf = (char*)malloc(need);
  if (qsim_plan_describe(p, buf, need, &need) != QSIM_OK || strstr(buf, "\"passes\"") == NULL) return 4;
  free(buf);
  qsim_plan_destroy(p);

  /* OpenQASM round trip of the same gate kinds */
  const char* text = "OPENQASM 2.0;\nqreg q[2];\nh q[0];\ncx q[0],q[1];\nry(pi/4) q[1];\n";
  qsim_gate pg[8];
  double params[8];
  int32_t ng = 0, np = 0, nq = 0;
  rc = qsim_parse_qasm(text, pg, 8, &ng, params, 8, &np, &nq);
  if (rc != QSIM_OK) {
    printf("parse failed: %d %s\n", rc, qsim_last_error());
    return 5;
  }
  printf("qasm %d %d %d %.17g\n", ng, np, nq, params[0]);
  char out[512];
  size_t out_need = 0;
  rc = qsim_export_qasm(pg, ng, nq, params, NULL, out, sizeof out, &out_need);
  if (rc != QSIM_OK || strstr(out, "ry(") == NULL) return 6;

  /* an invalid gate is reported with its code and a message */
  qsim_gate bad = {QSIM_RX, {5, -1}, {-1, -1}, 0};
  qsim_plan_t p2 = NULL;
  rc = qsim_plan(&bad, 1, 2, NULL, &p2);
  printf("error %d %s\n", rc, qsim_last_error());
  return (rc == QSIM_ERR_QUBIT && p2 == NULL) ? 0 : 7;
}
