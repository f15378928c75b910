/* Test driver: the FP64 oracle compiled with AddressSanitizer and
 * UndefinedBehaviorSanitizer runs a small failure-exercising tensile bar for
 * every damage model (none, Cockcroft-Latham, Johnson-Cook, GTN) through
 * plastic flow, damage and failure, with the rigid wall on.  Any out-of-bounds
 * access, use of freed memory or undefined arithmetic aborts with a report.
 * Compiled together with the oracle as one translation unit by
 * tests/test_oracle_sanitizers.py; test infrastructure only. */
#include "../oracle/tlsph_oracle.c"

#include <stdio.h>
#include <stdlib.h>

static double frand(uint64_t *s)
{
    /* xorshift64*: jitter for the driver's lattice only */
    *s ^= *s >> 12;
    *s ^= *s << 25;
    *s ^= *s >> 27;
    return (double)((*s * 2685821657736338717ULL) >> 11) * (1.0 / 9007199254740992.0);
}

static int run(int damage)
{
    const int nx = 4, ny = 4, nz = 14;
    const int64_t N = nx * ny * nz;
    const double d = 0.5e-3, h = 1.5 * d, rc = 2.0 * h;
    double *X = malloc(sizeof(double) * 3 * N), *vol = malloc(sizeof(double) * N);
    int32_t *mat = calloc(N, sizeof(int32_t));
    uint8_t *bcm = calloc(N, 1);
    double *bcv = calloc(3 * N, sizeof(double));
    uint64_t seed = 88172645463325252ULL;
    for (int64_t i = 0; i < N; ++i) {
        const int ix = (int)(i % nx), iy = (int)((i / nx) % ny), iz = (int)(i / (nx * ny));
        X[3 * i] = ix * d + 0.01 * d * (2 * frand(&seed) - 1);
        X[3 * i + 1] = iy * d + 0.01 * d * (2 * frand(&seed) - 1);
        X[3 * i + 2] = (iz + 0.5) * d + 0.01 * d * (2 * frand(&seed) - 1);
        vol[i] = d * d * d;
        if (iz < 2 || iz >= nz - 2) {
            bcm[i] = 1;
            bcv[3 * i + 2] = iz < 2 ? -20.0 : 20.0;
        }
    }
    const int64_t cap = N * N;
    int64_t *row_ptr = malloc(sizeof(int64_t) * (N + 1));
    int32_t *col = malloc(sizeof(int32_t) * cap);
    const int64_t nnz = orc_neighbors(N, X, rc, row_ptr, col, cap);
    double *L = malloc(sizeof(double) * 9 * N), *Linv = malloc(sizeof(double) * 9 * N);
    orc_shape_matrix(N, X, vol, row_ptr, col, h, L, Linv);

    orc_material m;
    memset(&m, 0, sizeof m);
    m.rho0 = 2700.0; m.E = 70e9; m.nu = 0.3; m.eos = damage == 3 ? 1 : 0; m.c0 = 5166.0; m.S_alpha = 1.4;
    m.Gamma0 = 2.0; m.A = 324e6; m.B = 114e6; m.n = 0.42; m.C = 0.002; m.epsdot0 = 1.0; m.damage = damage;
    m.Wcr = 1e6; m.D1 = 0.003; m.D2 = 0.003; m.D3 = -1.5;
    m.q1 = 1.5; m.q2 = 1.0; m.q3 = 2.25; m.fN = 0.04; m.eN = 0.3; m.sN = 0.1; m.fc = 0.15; m.fF = 0.25;
    double *f0 = calloc(N, sizeof(double));
    if (damage == 3)
        for (int64_t i = 0; i < N; ++i) f0[i] = 0.0008 + 0.0004 * frand(&seed);

    orc_system s;
    memset(&s, 0, sizeof s);
    s.N = N; s.X = X; s.vol = vol; s.mat_id = mat; s.bc_mask = bcm; s.bc_vel = bcv;
    s.row_ptr = row_ptr; s.col = col; s.Linv = Linv; s.mats = &m;
    s.u = calloc(3 * N, sizeof(double)); s.v = calloc(3 * N, sizeof(double)); s.F = calloc(9 * N, sizeof(double));
    s.sd = calloc(9 * N, sizeof(double)); s.sigma = calloc(9 * N, sizeof(double)); s.A = calloc(9 * N, sizeof(double));
    s.ep = calloc(N, sizeof(double)); s.epdot = calloc(N, sizeof(double)); s.dinit = calloc(N, sizeof(double));
    s.D = calloc(N, sizeof(double)); s.f = f0; s.e = calloc(N, sizeof(double));
    s.force = calloc(3 * N, sizeof(double));
    s.fail_step = calloc(N, sizeof(int32_t)); s.vh = calloc(3 * N, sizeof(double)); s.Fdot = calloc(9 * N, sizeof(double));
    orc_init_state(&s);
    orc_config c = { h, rc, 0.3 * d / 5907.6, 10.0, 1 };
    orc_step(&s, &c, 400);
    double epmax = 0.0;
    int64_t failed = 0;
    for (int64_t i = 0; i < N; ++i) {
        if (s.ep[i] > epmax) epmax = s.ep[i];
        failed += s.fail_step[i] >= 0;
    }
    printf("damage %d: N %lld nnz %lld max ep %.3e failed %lld status %u\n", damage, (long long)N, (long long)nnz,
           epmax, (long long)failed, s.status);
    free(X); free(vol); free(mat); free(bcm); free(bcv); free(row_ptr); free(col); free(L); free(Linv); free(f0);
    free(s.u); free(s.v); free(s.F); free(s.sd); free(s.sigma); free(s.A); free(s.ep); free(s.epdot); free(s.dinit);
    free(s.D); free(s.e); free(s.force); free(s.fail_step); free(s.vh); free(s.Fdot);
    return epmax > 0.0 ? 0 : 1;
}

int main(void)
{
    int rc = 0;
    for (int damage = 0; damage <= 3; ++damage) rc |= run(damage);
    return rc;
}
