/*
 * A plain-C user of the library (include/lift.h): ROF denoising with the
 * lifted relaxation (L = 2, Prop. 3), everything through the C ABI.
 *
 *   solve_rof <f.raw> <u.raw> <H> <W> <iters>
 *
 * f.raw holds H*W float32 values (row-major); the unlifted result is written
 * to u.raw in the same layout.  Prints the energies; exits 0 on success and
 * with the library's error code otherwise.
 */
#include <stdio.h>
#include <stdlib.h>

#include "lift.h"

static int fail(const char *what, int rc)
{
    fprintf(stderr, "%s: %s (%d)\n", what, lift_strerror(rc), rc);
    return rc ? rc : 1;
}

int main(int argc, char **argv)
{
    if (argc != 6) {
        fprintf(stderr, "usage: %s f.raw u.raw H W iters\n", argv[0]);
        return 1;
    }
    const int H = atoi(argv[3]), W = atoi(argv[4]), iters = atoi(argv[5]);
    const size_t n = (size_t)H * (size_t)W;
    float *f = (float *)malloc(n * sizeof(float));
    float *u = (float *)malloc(n * sizeof(float));
    if (!f || !u) return 1;
    FILE *in = fopen(argv[1], "rb");
    if (!in || fread(f, sizeof(float), n, in) != n) return 1;
    fclose(in);

    lift_spec spec = {0};
    spec.kind = LIFT_QUAD;
    spec.H = H;
    spec.W = W;
    spec.L = 2;
    spec.gamma_min = 0.0;
    spec.gamma_max = 1.0;
    spec.lambda = 0.2;
    spec.alpha = 1.0;
    spec.f = f;
    spec.data_on_host = 1;
    spec.check_every = 100;

    lift_handle h = NULL;
    int rc = lift_create(&spec, NULL, &h);
    if (rc != LIFT_OK) return fail("lift_create", rc);
    rc = lift_iterate(h, iters);
    if (rc != LIFT_OK) return fail("lift_iterate", rc);
    double primal = 0.0, dual = 0.0, enc = 0.0;
    rc = lift_energy(h, &primal, &dual, &enc);
    if (rc != LIFT_OK) return fail("lift_energy", rc);
    rc = lift_unlift(h, u, 1);
    if (rc != LIFT_OK) return fail("lift_unlift", rc);
    lift_destroy(h);

    FILE *out = fopen(argv[2], "wb");
    if (!out || fwrite(u, sizeof(float), n, out) != n) return 1;
    fclose(out);
    printf("%.10g %.10g %.10g\n", primal, dual, enc);
    free(f);
    free(u);
    return 0;
}
