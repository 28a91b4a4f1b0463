// Orders N compiled into the fused step kernel (one translation unit per order).  The three-plane
// ring of the new even class on a haloed 34 x 10 tile must fit in shared memory: 3 * n_even * 340 *
// 4 bytes (N = 9: 183,600).  The build reads this list: keep it a single line of X(n) entries.
#pragma once
#define RTPN_FUSED_ORDERS(X) X(1) X(3) X(5) X(7) X(9)
