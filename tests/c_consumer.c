/* A plain C99 consumer of the C ABI: includes logdet.h, links liblogdet.so and calls the
 * host-only entry points (no device work), so it runs without a GPU.  Prints one line of
 * results for tests/test_c_consumer.py to check; exits nonzero on the first failure. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include "logdet.h"

#define CHECK(cond)                                                       \
    do {                                                                  \
        if (!(cond)) {                                                    \
            fprintf(stderr, "failed: %s (%s)\n", #cond, ld_last_error()); \
            return 1;                                                     \
        }                                                                 \
    } while (0)

int main(void) {
    CHECK(ld_abi_version() == LD_ABI_VERSION);

    ld_options opt;
    CHECK(ld_default_options(&opt) == LD_OK);
    CHECK(opt.precision == LD_FP64);

    /* distance-2 colouring of a 5-point 8 x 8 Dirichlet grid */
    int32_t dims[3] = {8, 8, 1};
    int32_t colour[64];
    int32_t nc = 0;
    CHECK(ld_colour_grid(LD_STENCIL_2D5, dims, 0, 2, colour, &nc) == LD_OK);
    CHECK(nc >= 5 && nc <= 64);

    /* quadrature nodes on [0.5, 8.5] and their certificate */
    double sigma[2 * 20], alpha[2 * 20], cert = 1.0;
    CHECK(ld_hht_nodes(0.5, 8.5, 20, sigma, alpha, &cert) == LD_OK);
    CHECK(cert < 1e-12);

    /* spectral interval of the 1D chain kappa^2 I - Lap (n = 50, kappa^2 = 0.3) as CSR */
    enum { N = 50 };
    int64_t rowptr[N + 1];
    int32_t colidx[3 * N];
    double val[3 * N];
    int64_t e = 0;
    for (int i = 0; i < N; ++i) {
        rowptr[i] = e;
        if (i > 0) { colidx[e] = i - 1; val[e++] = -1.0; }
        colidx[e] = i; val[e++] = 2.3;
        if (i + 1 < N) { colidx[e] = i + 1; val[e++] = -1.0; }
    }
    rowptr[N] = e;
    double lmin = 0.0, lmax = 0.0;
    CHECK(ld_csr_bounds(N, rowptr, colidx, val, 1.0, &lmin, &lmax) == LD_OK);
    const double exact_min = 0.3 + 2.0 - 2.0 * cos(M_PI / (N + 1));
    CHECK(lmin > 0.0 && lmin <= exact_min && lmax >= 4.3 - 1e-12);

    /* a two-triangle mesh of the unit square: query nnz, then fill */
    const double xy[8] = {0, 0, 1, 0, 0, 1, 1, 1};
    const int64_t tri[6] = {0, 1, 3, 0, 3, 2};
    int64_t nnz = 0;
    CHECK(ld_spde_fem_csr(4, xy, 2, tri, 1.0, 1, 1.0, 0, NULL, NULL, NULL, &nnz) == LD_OK);
    int64_t rp[5];
    int32_t *ci = malloc((size_t)nnz * sizeof(int32_t));
    double *vv = malloc((size_t)nnz * sizeof(double));
    CHECK(ci && vv);
    CHECK(ld_spde_fem_csr(4, xy, 2, tri, 1.0, 1, 1.0, nnz, rp, ci, vv, &nnz) == LD_OK);
    double total = 0.0;   /* 1^T (kappa^2 C + G) 1 = kappa^2 |domain| = 1 */
    for (int64_t k = 0; k < nnz; ++k) total += vv[k];
    CHECK(fabs(total - 1.0) < 1e-14);

    /* errors come back as status codes with a message */
    CHECK(ld_hht_nodes(2.0, 1.0, 20, sigma, alpha, &cert) == LD_EINVAL);
    CHECK(ld_last_error()[0] != '\0');

    printf("ok colours=%d cert=%.3g lmin=%.6g lmax=%.6g nnz=%lld total=%.15g\n", (int)nc, cert, lmin,
           lmax, (long long)nnz, total);
    free(ci);
    free(vv);
    return 0;
}
