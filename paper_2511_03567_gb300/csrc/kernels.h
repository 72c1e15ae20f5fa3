// Launchers of the elementwise / setup kernels (kernels.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

void launch_scatter(double* dst, const double* src, const int64_t* idx, const int64_t* idx2,
                    int64_t n, cudaStream_t s);
void launch_gather(double* dst, const double* src, const int64_t* idx, const int64_t* idx2,
                   int64_t n, cudaStream_t s);
void launch_fock(double* F, const double* h, const double* eri, const double* g1, const Dims& d,
                 cudaStream_t s);
void launch_e0(double* out, const double* h, const double* F, const double* eri, const double* g1,
               const double* l2, const Dims& d, cudaStream_t s);
void launch_cumulant2(double* L2, double* D2, double* G, double* E, const double* g1,
                      const double* g2, int a, int given, cudaStream_t s);
void launch_direct3(double* D3, const double* L3, int a, cudaStream_t s);
void launch_update(const double* T, const double* X, double* Tn, double* Err, const double* eps,
                   const Dims& d, double s, double* maxdt, cudaStream_t st);
void launch_dots(double* dots, const double* enew, const double* hist, int64_t n, int m,
                 int64_t ld, cudaStream_t st);
void launch_diis_solve(const double* gram, double* coef, int m, int* status, cudaStream_t st);
void launch_extrapolate(double* T, const double* vecs, const double* coef, const int* status,
                        int m, int newest, int64_t n, int64_t ld, cudaStream_t st);
// Cyclic Jacobi eigen-decomposition of one symmetric block (overwritten)
// into columns of U at (off, off); *d_sweeps (device) receives the sweeps or
// -1 if the sweep limit was reached unconverged.  Returns the launch status.
cudaError_t run_jacobi(double* Ablk, double* V, int n, double* U, int n_full, int off, int* d_sweeps,
                       cudaStream_t s);
void launch_energy_out(double* out, const double* acc, double e0, cudaStream_t s);
// y += x over n elements
void launch_add(double* y, const double* x, int64_t n, cudaStream_t s);
void launch_adj_y(const double* Lam, double* Yraw, double* Ytil, const double* eps, const Dims& d, double s,
                  cudaStream_t st);
void launch_adj_update(const double* Lam, const double* Yraw, const double* GT, double* Ln, double* Err,
                       const double* eps, const Dims& d, double* maxd, cudaStream_t st);
void launch_adj_eps(const double* Lam, const double* T, const double* X, const double* eps, const Dims& d,
                    double s, double* geps, double* dEds, cudaStream_t st);
// gFt, gh [n][n]; geri gets the Fock/E0 chain and is then pair-symmetrised
void launch_adj_chain(double* geri, const double* gF, const double* geps, const double* g1, const double* l2,
                      const Dims& d, double* gFt, double* gh, cudaStream_t st);
