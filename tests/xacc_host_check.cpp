// Host build of the exact accumulator's merge and final rounding
// (paper_2108_10591_gb300/csrc/xacc.cuh, whose 192-bit part is host-capable),
// for CPU tests against exact rational arithmetic.
#define __host__
#define __device__
#define __forceinline__ inline
#include "xacc.cuh"

extern "C" {

double xh_round(int e, unsigned long long w2, unsigned long long w1, unsigned long long w0) {
    bcs::XAcc a{e, w2, w1, w0};
    return bcs::xa_round(a);
}

// a += b; w[] = {w2, w1, w0}
void xh_merge(int ea, const unsigned long long* wa, int eb, const unsigned long long* wb, int* e,
              unsigned long long* w) {
    bcs::XAcc a{ea, wa[0], wa[1], wa[2]};
    const bcs::XAcc b{eb, wb[0], wb[1], wb[2]};
    bcs::xa_merge(a, b);
    *e = a.e;
    w[0] = a.w2;
    w[1] = a.w1;
    w[2] = a.w0;
}

int xh_empty() { return bcs::kXaEmpty; }
int xh_nan() { return bcs::kXaNaN; }
}
