// (order, tile x, tile y, tile z, stage buffers, TMA box length step) variants of the
// TMA-staged kernel, one translation unit each, instantiated for FP32 and BF16 storage where the
// stage ring fits shared memory (the deeper rings fit BF16 only).  The default for a grid is the
// first listed variant that fits and whose width divides nx.  At most one entry per (order, tile,
// depth).  The build reads this list: keep it a single line of X(...) entries.
#pragma once
#define RTPN_STAGE_VARIANTS(X) X(39, 40, 2, 2, 2, 1) X(39, 40, 2, 2, 4, 1) X(39, 32, 2, 2, 3, 1) X(29, 32, 2, 2, 3, 1) X(29, 40, 2, 2, 2, 1) X(19, 32, 2, 2, 3, 1) X(19, 40, 2, 2, 2, 1) X(15, 32, 3, 3, 3, 1) X(15, 32, 2, 2, 3, 1) X(15, 32, 2, 2, 4, 1) X(15, 16, 4, 4, 4, 1) X(15, 48, 2, 2, 4, 1) X(15, 64, 2, 2, 3, 1) X(7, 32, 2, 2, 4, 1)
