// Orders N compiled into register-window kernels (one translation unit per order and class).
// The build reads this list: keep it a single line of X(n) entries.
#pragma once
#define RTPN_WINDOW_ORDERS(X) X(1) X(3) X(5) X(7) X(9) X(15) X(39)
