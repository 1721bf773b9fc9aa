// Compile-time dispatch over (dimension, level degree).
#pragma once

#define EMG_DISPATCH_DP(dim, p, FN)        \
    switch ((dim) * 8 + (p)) {             \
        case 16: FN(2, 0); break;          \
        case 17: FN(2, 1); break;          \
        case 18: FN(2, 2); break;          \
        case 19: FN(2, 3); break;          \
        case 20: FN(2, 4); break;          \
        case 24: FN(3, 0); break;          \
        case 25: FN(3, 1); break;          \
        case 26: FN(3, 2); break;          \
        case 27: FN(3, 3); break;          \
        case 28: FN(3, 4); break;          \
        default:                           \
            c->err = "unsupported (dim, p)"; \
            return EMG_ERR_ARG;            \
    }

namespace emg {
struct U5 {
    double v[5];
};
}  // namespace emg
