// Masked tensor-window step kernels for the rule of 8 points per axis,
// window widths 6..7 (every cell-offset pattern of each): the single-field
// step, the persistent march and their shared-memory opt-in.  The kernels are
// in fk_window.cuh; a few widths per translation unit keep the parallel
// build short.
#include "fk_window.cuh"

FK_DEFINE_MASKED_QW(8, 6)
FK_DEFINE_MASKED_QW(8, 7)
