// hbe_aux.h -- launchers of the non-stage kernels (hbe_aux.cu).
#pragma once
#include "hbe_common.cuh"

namespace hbe {

// prec here is the storage class of the state: 0 = double, 1 = float.
cudaError_t launch_pack(int prec, const double *src, void *hi, void *lo, int N, int pitch, int hx,
                        int periodic, int z_begin, int z_count, cudaStream_t st);
cudaError_t launch_unpack(int prec, const void *hi, const void *lo, double *dst, int N, int pitch,
                          int hx, int z_begin, int z_count, cudaStream_t st);
cudaError_t launch_bumps(int prec, void *hi, void *lo, int N, int pitch, int hx, int periodic,
                         double h, int nb, const double *d_prm, cudaStream_t st);
// The step coefficients of steps 0 .. K-1 of the coming batch of each context
// (Desc::coef); launched before the batch's stage kernels.
cudaError_t launch_coef(Desc *descs, const int *ndesc, int max_desc, int K, cudaStream_t st);
cudaError_t launch_advance(Desc *descs, const int *ndesc, int max_desc, int K, cudaStream_t st);
// Periodic ghost copies of the fields stage `stage` (1..6, 5 and 6 the fused
// pairs) wrote for step k of the batch; contexts that are not periodic or did
// not take the step are skipped.  `blocks` blocks of 256 threads per context.
bool stage_needs_wrap(int stage);
cudaError_t launch_wrap(Desc *descs, const int *ndesc, int max_desc, int k, int stage,
                        int blocks, cudaStream_t st);
// Halo planes of a z-slab decomposition after stage pair `stage` of step k of
// a replay: 5 -> G1, G2; 6 -> phi, psi of the new state.  One copy per entry
// of `copies` (n entries); a copy whose source did not take the step is skipped.
cudaError_t launch_halo(const Desc *descs, const HaloCopy *copies, int n, int k, int stage,
                        cudaStream_t st);
cudaError_t launch_set_run(Desc *d, long long add_steps, double t0, double dt, double thr,
                           int reset, cudaStream_t st);
cudaError_t launch_signpack(int prec, const void *hi, const void *lo, int N, int pitch, int hx,
                            double eps, uint32_t *pos, uint32_t *neg, unsigned long long *maxbits,
                            cudaStream_t st);
cudaError_t launch_ccl(const uint32_t *mask, int N, int periodic, int *labels,
                       unsigned long long *count, unsigned *err, cudaStream_t st);

int analysis_blocks();
cudaError_t launch_analysis(int prec, const void *phi, const void *phlo, const void *psi,
                            const void *pslo, int N, int pitch, int hx, int periodic,
                            double inv_h2, double mcoef, double eps, double *part, double *out,
                            cudaStream_t st);

}  // namespace hbe
