// Masked tensor-window step kernels for the rule of 4 points per axis
// (window widths 3..9, every cell-offset pattern of each); the kernel is in
// fk_window.cuh.  One translation unit per rule size keeps the parallel
// build short.
#include "fk_window.cuh"

FK_DEFINE_MASKED_Q(4)
