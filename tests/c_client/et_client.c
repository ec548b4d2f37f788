/* A plain C client of the library's C ABI (include/et.h): no Python, no
 * PyTorch.  It allocates the workspace with the CUDA runtime, builds a small
 * diffusion field and seed on the host, advances the grid through the host
 * entry points and prints the final state and record for the test to compare.
 *
 * usage: et_client nx ny nz nsteps precision(0 f64, 1 f32, 2 df64) out.bin
 * out.bin receives the nx*ny*nz final densities (FP64) followed by the
 * record's mass, umin, umax, s, m. */
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>

#include "et.h"

static int check(et_status st, et_grid* g, const char* what) {
    if (st != ET_OK) {
        fprintf(stderr, "%s: %s (%s)\n", what, et_status_string(st), et_last_error(g));
        return 1;
    }
    return 0;
}

int main(int argc, char** argv) {
    if (argc != 7) {
        fprintf(stderr, "usage: et_client nx ny nz nsteps precision out.bin\n");
        return 2;
    }
    const int nx = atoi(argv[1]), ny = atoi(argv[2]), nz = atoi(argv[3]), nsteps = atoi(argv[4]);
    const et_precision prec = (et_precision)atoi(argv[5]);
    const long n = (long)nx * ny * nz;
    double* D = (double*)malloc(sizeof(double) * n);
    double* u = (double*)malloc(sizeof(double) * n);
    if (!D || !u) return 2;
    /* a sphere of tissue (D = 0.13, 0.013 in an outer shell) in air, seed at the centre */
    const double cx = 0.5 * (nx - 1), cy = 0.5 * (ny - 1), cz = 0.5 * (nz - 1);
    const double r = 0.45 * (nx < ny ? (nx < nz ? nx : nz) : (ny < nz ? ny : nz));
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const long p = i + (long)nx * (j + (long)ny * k);
                const double dx = i - cx, dy = j - cy, dz = k - cz;
                const double d2 = dx * dx + dy * dy + dz * dz;
                D[p] = d2 < 0.36 * r * r ? 0.13 : (d2 < r * r ? 0.013 : 0.0);
                u[p] = d2 < 4.0 ? 0.8 : 0.0;
            }
    const size_t bytes = et_workspace_bytes(nx, ny, nz, prec);
    void* ws = NULL;
    if (bytes == 0 || cudaMalloc(&ws, bytes) != cudaSuccess) {
        fprintf(stderr, "workspace allocation failed\n");
        return 1;
    }
    et_grid* g = NULL;
    if (check(et_create_grid(nx, ny, nz, 1.0, prec, ws, bytes, NULL, &g), NULL, "et_create_grid")) return 1;
    if (check(et_set_coeffs_host(g, D, 0.025, ET_OP_CONSERVATIVE, ET_SCHEME_ROSENBROCK, NULL), g, "et_set_coeffs_host"))
        return 1;
    et_step_info rec;
    if (check(et_run_host(g, u, 7.3, nsteps, &rec), g, "et_run_host")) return 1;
    FILE* f = fopen(argv[6], "wb");
    if (!f) return 1;
    const double tail[5] = {rec.mass, rec.umin, rec.umax, (double)rec.s, (double)rec.m};
    fwrite(u, sizeof(double), (size_t)n, f);
    fwrite(tail, sizeof(double), 5, f);
    fclose(f);
    printf("et_client: grid %dx%dx%d, %d steps, mass %.12g, s %d, m %d\n", nx, ny, nz, nsteps, rec.mass, rec.s,
           rec.m);
    et_destroy(g);
    cudaFree(ws);
    free(D);
    free(u);
    return 0;
}
