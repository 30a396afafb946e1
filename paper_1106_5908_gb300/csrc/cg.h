// Vector kernels of the CG solvers (device scalars live in a small array `sc`).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace spmv {

// Slots of the device scalar array.
enum : int { kScRho = 0, kScPQ = 1, kScAlpha = 2, kScBeta = 3, kScNorm = 4, kScCount = 8 };
// Scalar steps applied after a reduction.
enum : int { kOpStore = 0, kOpAlpha = 1, kOpBeta = 2 };

// Where a reduction ends: partials (one per block), the ticket counting
// finished blocks (zero between launches) and the scalar step op applied to
// the sum, written to sc[dst] (kOpStore) or to the CG scalars.
struct RedOut {
    double *partials;
    unsigned int *ticket;
    double *sc;
    int op;
    int dst;
};

// doubles of the reduction work array (partials and the ticket word; zero it once)
int cg_partials_len();
// The reduction target in that work array for a launch of at most
// cg_partials_cap() blocks.
RedOut cg_red_out(double *partials, double *sc, int op, int dst);
int cg_partials_cap();
// sc[dst] = a.b (op kOpStore) or alpha = sc[rho]/(a.b) (op kOpAlpha).  FP64 accumulation.
cudaError_t cg_dot(const void *a, int ak, const void *b, int bk, int64_t n, double *partials,
                   double *sc, int op, int dst, cudaStream_t s);
// d += alpha p, r -= alpha q (FP32), then beta = r.r / rho, rho = r.r.
cudaError_t cg_update32(float *d, float *r, const float *p, const float *q, int64_t n,
                        double *partials, double *sc, cudaStream_t s);
// x += alpha p, r -= alpha q (FP64), then beta = r.r / rho, rho = r.r.
cudaError_t cg_update64(double *x, double *r, const double *p, const double *q, int64_t n,
                        double *partials, double *sc, cudaStream_t s);
// p = r + beta p
cudaError_t cg_direction(void *p, const void *r, int k, const double *sc, int64_t n, cudaStream_t s);
cudaError_t cg_scale_to32(const double *r64, float *r32, double scale, int64_t n, cudaStream_t s);
cudaError_t cg_axpy_64_32(double *x, const float *d, double scale, int64_t n, cudaStream_t s);

}  // namespace spmv
