// Dispatch of the masked tensor-window step kernels (fk_window.cuh) by rule
// size, and the host-side helpers the plan uses to size and select them.
#include <cuda_runtime.h>

#include "fk_internal.h"

size_t fk_step2dm_smem(int ly, int lx) {
  // point constants, then pair records (16 B + 8 B) and u^{n+1} (4 B) per staged node
  return (size_t)FK_MAXQ_2D * 16 + (size_t)ly * lx * (16 + 8 + 4);
}

int fk_step2dm_lx(int hx, int w) { return 32 + 2 * hx + 2 + ((w + 1) / 2 * 2 - w); }

bool fk_masked_available(int q, int w) {
  return (q == 4 || q == 6 || q == 8) && w >= 3 && w <= 9;
}

int fk_masked_pattern(int q, int w, const int* m) {
  if (!fk_masked_available(q, w)) return -1;
  for (int k = 0; k < fk_npat(q, w); ++k) {
    bool same = true;
    for (int i = 0; i < q && same; ++i) same = fk_mpat(q, w, k, i) == m[i];
    if (same) return k;
  }
  return -1;
}

// (each macro expands to one test per (Q, W) of FK_MASKED_ALL)
cudaError_t fk_launch_step2dm(const Step2D<float>& a, int q, cudaStream_t s) {
#define FK_CASE(QQ, WW) \
  if (q == QQ && a.win == WW) return fk_launch_step2dm_q##QQ##w##WW(a, s);
  FK_MASKED_ALL(FK_CASE)
#undef FK_CASE
  return cudaErrorInvalidValue;
}

cudaError_t fk_prepare_masked_kernels(int q) {
  cudaError_t e = cudaSuccess;
#define FK_CASE(QQ, WW) \
  if (q == QQ && e == cudaSuccess) e = fk_prepare_masked_q##QQ##w##WW();
  FK_MASKED_ALL(FK_CASE)
#undef FK_CASE
  return e;
}

cudaError_t fk_launch_march2dm(const Step2D<float>& a, const MaskedMarch& m, int q,
                               cudaStream_t s) {
#define FK_CASE(QQ, WW) \
  if (q == QQ && a.win == WW) return fk_launch_march2dm_q##QQ##w##WW(a, m, s);
  FK_MASKED_ALL(FK_CASE)
#undef FK_CASE
  return cudaErrorInvalidValue;
}

bool fk_march2dm_fits(const Step2D<float>& a, int q) {
#define FK_CASE(QQ, WW) \
  if (q == QQ && a.win == WW) return fk_march2dm_fits_q##QQ##w##WW(a);
  FK_MASKED_ALL(FK_CASE)
#undef FK_CASE
  return false;
}
