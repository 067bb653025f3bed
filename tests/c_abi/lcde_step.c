/* A C caller of libmmfd with no Python or PyTorch: a two-level D2Q9 linear CDE on a periodic
 * nx x ny grid, FP64 storage, the library's own cudaMalloc allocator and the default stream.
 * Reads phi0 (nx*ny doubles, x fastest) from argv[1], advances argv[4] steps and writes the
 * field to argv[2]; prints the field sum before and after (FP64 reductions).
 * usage: lcde_step in.bin out.bin nx ny steps */
#include <stdio.h>
#include <stdlib.h>

#include "mmfd.h"

#define CHECK(call)                                                                          \
    do {                                                                                     \
        int rc_ = (call);                                                                    \
        if (rc_ != MMFD_OK) {                                                                \
            fprintf(stderr, "%s failed: %s (%s)\n", #call, mmfd_strerror(rc_), mmfd_last_error()); \
            return 1;                                                                        \
        }                                                                                    \
    } while (0)

int main(int argc, char** argv) {
    if (argc != 6) {
        fprintf(stderr, "usage: %s in.bin out.bin nx ny steps\n", argv[0]);
        return 2;
    }
    const long long nx = atoll(argv[3]), ny = atoll(argv[4]), steps = atoll(argv[5]);
    const size_t n = (size_t)(nx * ny);
    double* phi = (double*)malloc(n * sizeof(double));
    if (!phi) return 1;
    FILE* f = fopen(argv[1], "rb");
    if (!f || fread(phi, sizeof(double), n, f) != n) return 1;
    fclose(f);

    mmfd_desc d;
    CHECK(mmfd_desc_init(&d));
    d.pde = MMFD_LCDE;
    d.lattice = MMFD_D2Q9;
    d.levels = 2;
    d.dim = 2;
    d.n[0] = nx;
    d.n[1] = ny;
    d.n[2] = 1;
    d.dt = 1.0;
    d.dx[0] = d.dx[1] = 1.0;
    d.K[0][0] = 0.02;
    d.K[0][1] = d.K[1][0] = 0.005;
    d.K[1][1] = 0.01;
    d.u[0] = 0.1;
    d.u[1] = 0.05;
    d.storage = MMFD_FP64;   /* targets (a_0, A10, A11, A21, A22) = (0, -1, -1, 0, 1/2) by default */

    mmfd_solver* s = NULL;
    CHECK(mmfd_create(&d, &s));
    const void* in[1] = {phi};
    CHECK(mmfd_set_fields(s, 0, in, MMFD_HOST, MMFD_DT_F64));
    double m0 = 0.0, m1 = 0.0;
    CHECK(mmfd_reduce(s, MMFD_RED_SUM, &m0));
    CHECK(mmfd_step(s, steps));
    CHECK(mmfd_reduce(s, MMFD_RED_SUM, &m1));
    void* out[1] = {phi};
    CHECK(mmfd_fields(s, 0, out, MMFD_HOST, MMFD_DT_F64));
    mmfd_info_t info;
    CHECK(mmfd_get_info(s, &info));
    CHECK(mmfd_destroy(s));

    f = fopen(argv[2], "wb");
    if (!f || fwrite(phi, sizeof(double), n, f) != n) return 1;
    fclose(f);
    printf("kernel %s mass %.17g %.17g\n", info.kernel, m0, m1);
    free(phi);
    return 0;
}
