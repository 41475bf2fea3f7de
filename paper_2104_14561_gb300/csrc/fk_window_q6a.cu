// Masked tensor-window step kernels for the rule of 6 points per axis,
// window widths 3..6 (every cell-offset pattern of each): the single-field
// step, the persistent march and their shared-memory opt-in.  The kernels are
// in fk_window.cuh; a few widths per translation unit keep the parallel
// build short.
#include "fk_window.cuh"

FK_DEFINE_MASKED_QW(6, 3)
FK_DEFINE_MASKED_QW(6, 4)
FK_DEFINE_MASKED_QW(6, 5)
FK_DEFINE_MASKED_QW(6, 6)
