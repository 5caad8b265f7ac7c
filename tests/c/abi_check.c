/* A plain C99 client of include/chhs.h: it compiles the header as C and
 * makes the calls that need no GPU (defaults, the workspace size and the
 * argument checks of chhs_create, which return before any CUDA call).
 * Exit status 0 when every check holds; each failed check prints a line. */
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "chhs.h"

static int failures = 0;

static void check(int ok, const char* what) {
    if (!ok) {
        printf("FAILED: %s\n", what);
        ++failures;
    }
}

int main(void) {
    chhs_opts o;
    int n2[3] = {64, 64, 1}, n3[3] = {32, 32, 32}, odd[3] = {1, 64, 1};
    chhs_t* run = (chhs_t*)&o; /* any non-NULL value: an error must reset it */
    size_t w2, w3;

    check(chhs_default_opts(&o) == CHHS_OK, "default opts");
    check(o.nu1 == 2 && o.nu2 == 2 && o.coarsest == 2 && o.tol == 1e-10 && o.precision == 0 &&
              o.max_factor == 50.0 && o.coarsest_f64 == 0 && o.f64_residual == 0 && o.max_inner == 3,
          "default values");
    check(chhs_default_opts(NULL) == CHHS_ERR_INVALID_ARG, "default opts NULL");

    w2 = chhs_workspace_bytes(2, n2, NULL);
    w3 = chhs_workspace_bytes(3, n3, &o);
    check(w2 > 0 && w3 > w2, "workspace sizes");
    check(chhs_workspace_bytes(2, odd, NULL) == 0, "workspace of a bad size");

    check(chhs_create(2, odd, 0.1, 0.05, 1.0, 0.01, NULL, NULL, &run) == CHHS_ERR_INVALID_ARG && run == NULL,
          "create with an extent < 2");
    run = (chhs_t*)&o;
    check(chhs_create(2, n2, 0.1, 0.05, -1.0, 0.01, NULL, NULL, &run) == CHHS_ERR_INVALID_ARG && run == NULL,
          "create with gamma < 0");
    run = (chhs_t*)&o;
    check(chhs_create(2, n2, NAN, 0.05, 1.0, 0.01, NULL, NULL, &run) == CHHS_ERR_INVALID_ARG && run == NULL,
          "create with h NaN");
    o.precision = 3;
    run = (chhs_t*)&o;
    check(chhs_create(2, n2, 0.1, 0.05, 1.0, 0.01, &o, NULL, &run) == CHHS_ERR_INVALID_ARG && run == NULL,
          "create with a bad precision");

    check(chhs_step(NULL, 1, NULL, NULL) == CHHS_ERR_INVALID_ARG, "step on NULL");
    check(chhs_num_levels(NULL) == 0, "levels of NULL");
    check(strcmp(chhs_last_error(NULL), "NULL handle") == 0, "last error of NULL");
    chhs_destroy(NULL);
    chhs_server_destroy(NULL);

    if (failures == 0) printf("abi_check: ok\n");
    return failures == 0 ? 0 : 1;
}
