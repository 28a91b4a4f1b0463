// (order, tile x, tile y, tile z, stage buffers) variants of the TMA-staged kernel, one translation
// unit each.  The build reads this list: keep it a single line of X(...) entries.
#pragma once
#define RTPN_STAGE_VARIANTS(X) X(39, 40, 2, 2, 2) X(39, 32, 2, 2, 3) X(15, 32, 4, 2, 4) X(7, 32, 4, 2, 4)
