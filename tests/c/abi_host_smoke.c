/* Plain C99 client of the C ABI: host-only calls (planning, host quasienergies, argument
 * errors), no device and no Python.  Exit status 0 when every check holds; each failure prints
 * one line.  Built and run by tests/test_c_abi.py. */
#include <complex.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "floquet.h"

static int failures = 0;

#define CHECK(cond, ...)            \
  do {                              \
    if (!(cond)) {                  \
      printf("FAIL: " __VA_ARGS__); \
      printf("\n");                 \
      ++failures;                   \
    }                               \
  } while (0)

int main(void) {
  /* a 4-site tridiagonal problem with a cosine drive: host planning fills L, R, the bounds */
  double d[4] = {0.0, 1.0, 2.0, 3.0}, off[3] = {-1.0, -1.0, -1.0}, h1[4] = {-1.5, -0.5, 0.5, 1.5};
  fq_problem p;
  memset(&p, 0, sizeof p);
  p.n = 4;
  p.format = FQ_TRIDIAG;
  p.h0 = d;
  p.h0_off = off;
  p.h1 = h1;
  p.period = 2.0 * M_PI / 3.0;
  p.steps = 20;
  p.drive_kind = FQ_DRIVE_COS;
  p.f_ac = 1.5;
  p.omega = 3.0;
  p.precision = FQ_FP32;
  fq_plan_info info;
  double a[64];
  fq_status st = floquet_plan_inspect(&p, &info, a, 64);
  CHECK(st == FQ_OK, "floquet_plan_inspect: status %d (%s)", (int)st, floquet_last_error());
  CHECK(info.n == 4 && info.steps == 20 && info.L >= 1 && info.L < 64, "info: n %d steps %d L %d", info.n,
        info.steps, info.L);
  CHECK(info.e_min < info.e_max && info.R > 0.0, "bounds [%g, %g], R %g", info.e_min, info.e_max, info.R);
  CHECK(fabs(info.R - info.h * 0.5 * (info.e_max - info.e_min)) <= 1e-14 * info.R, "R = h Delta E");
  /* a_0 = J_0(R), a_l = 2 J_l(R): the sum rule J_0 + 2 sum_k J_2k = 1 over the even weights */
  double sum = 0.0;
  for (int l = 0; l <= info.L; l += 2) sum += a[l];
  CHECK(fabs(sum - 1.0) < 1e-12, "even Bessel weights sum to %.17g", sum);

  /* argument errors come back as statuses with a message */
  p.steps = 0;
  st = floquet_plan_inspect(&p, &info, NULL, 0);
  CHECK(st == FQ_EINVAL && strlen(floquet_last_error()) > 0, "steps = 0: status %d", (int)st);
  p.steps = 20;
  p.omega = NAN;
  st = floquet_plan_inspect(&p, &info, NULL, 0);
  CHECK(st == FQ_EINVAL, "omega = NaN: status %d", (int)st);

  /* host quasienergies of a diagonal U_T with known phases, as C99 complex numbers */
  double complex u[9] = {0};
  const double th[3] = {0.7, -2.1, 3.0};
  for (int k = 0; k < 3; ++k) u[4 * k] = cexp(-I * th[k]);
  double eps[3];
  double complex states[9];
  st = floquet_quasienergies(u, 3, 2.0, eps, states);
  CHECK(st == FQ_OK, "floquet_quasienergies: status %d (%s)", (int)st, floquet_last_error());
  const double want[3] = {-2.1 / 2.0, 0.7 / 2.0, 3.0 / 2.0};
  for (int k = 0; k < 3; ++k) CHECK(fabs(eps[k] - want[k]) < 1e-14, "eps[%d] = %.17g, want %.17g", k, eps[k], want[k]);
  /* the state of the lowest quasienergy is basis vector 1 up to a phase */
  CHECK(fabs(cabs(states[1]) - 1.0) < 1e-14, "|state_0[1]| = %.17g", cabs(states[1]));
  st = floquet_quasienergies(u, 3, -1.0, eps, NULL);
  CHECK(st == FQ_EINVAL, "period < 0: status %d", (int)st);

  /* workspace queries on a NULL plan are 0, not a crash */
  CHECK(floquet_workspace_size(NULL, 4) == 0, "workspace size of NULL plan");
  CHECK(floquet_defect_workspace_size(0) == 0 && floquet_defect_workspace_size(4) > 0, "defect workspace sizes");
  if (failures == 0) printf("ok\n");
  return failures == 0 ? 0 : 1;
}
