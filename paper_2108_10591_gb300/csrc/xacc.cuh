// Exact, order-independent inner-product accumulation on the integer pipes.
//
// Every product x_j y_j is formed exactly as an integer (53 x 53 -> 106 bits
// for FP64 operands, 24 x 24 -> 48 bits for FP32) with a power-of-two weight,
// and added into a 128-bit two's-complement fixed-point window
//     value = w * 2^e.
// The window is anchored so that the largest term seen so far ends at bit
// kTop (18 bits of headroom above it); when a larger term arrives the window
// slides up, dropping bits more than 2^-110 below the largest term.  Partial
// accumulators from different threads and CTAs are aligned to the larger
// anchor and added as integers.  The final value is rounded once to FP64,
// nearest even.  Up to the dropped bits (2^-110 relative to the largest term,
// far below the 2^-53 rounding unit unless the sum cancels by more than ~2^50)
// the result is the correctly rounded inner product, independent of the order
// in which terms and partials were combined.  No FP64 arithmetic is used, so
// the scarce FP64 units of the GPU stay with the recurrences and the SpMV.
#pragma once
#include <stdint.h>

namespace bcs {

constexpr int kXaTop = 110;              // anchor headroom: terms end at or below bit kXaTop
constexpr int kXaEmpty = -(1 << 29);     // e of an accumulator with no terms
constexpr int kXaNaN = (1 << 29);        // e of an accumulator that saw a NaN/Inf operand

struct XAcc {
    int e;
    unsigned long long hi, lo;  // 128-bit two's complement
};

__host__ __device__ __forceinline__ int xa_clz64(unsigned long long v) {
#ifdef __CUDA_ARCH__
    return __clzll((long long)v);
#else
    return v ? __builtin_clzll(v) : 64;
#endif
}
__host__ __device__ __forceinline__ unsigned long long xa_mulhi64(unsigned long long a, unsigned long long b) {
#ifdef __CUDA_ARCH__
    return __umul64hi(a, b);
#else
    return (unsigned long long)(((unsigned __int128)a * b) >> 64);
#endif
}

__host__ __device__ __forceinline__ void xa_init(XAcc& a) {
    a.e = kXaEmpty;
    a.hi = 0;
    a.lo = 0;
}

// arithmetic shift right of (hi, lo) by d >= 0
__host__ __device__ __forceinline__ void xa_sra(unsigned long long& hi, unsigned long long& lo, int d) {
    if (d <= 0) return;
    const long long sh = (long long)hi;
    if (d >= 128) {
        hi = lo = (unsigned long long)(sh >> 63);
    } else if (d >= 64) {
        lo = (unsigned long long)(sh >> (d - 64));
        hi = (unsigned long long)(sh >> 63);
    } else {
        lo = (lo >> d) | (hi << (64 - d));
        hi = (unsigned long long)(sh >> d);
    }
}

__host__ __device__ __forceinline__ void xa_add128(unsigned long long& hi, unsigned long long& lo,
                                                   unsigned long long th, unsigned long long tl) {
    const unsigned long long l = lo + tl;
    hi = hi + th + (l < lo ? 1ull : 0ull);
    lo = l;
}

// Keep |w| < 2^124 so that adding two accumulators never overflows.
__host__ __device__ __forceinline__ void xa_norm(XAcc& a) {
    const long long t = (long long)a.hi >> 60;  // 0 or -1 when |w| < 2^124
    if (t != 0 && t != -1) {
        xa_sra(a.hi, a.lo, 4);
        a.e += 4;
    }
}

// Add the term (ph:pl) * 2^e (unsigned magnitude, 1 <= ph:pl < 2^107), negated if neg.
__host__ __device__ __forceinline__ void xa_add_term(XAcc& a, unsigned long long ph, unsigned long long pl, int e,
                                                     bool neg) {
    const int len = ph ? 128 - xa_clz64(ph) : 64 - xa_clz64(pl);
    const int top = e + len;
    if (a.e == kXaNaN) return;
    if (a.e == kXaEmpty) {
        a.e = top - kXaTop;
    } else if (top > a.e + kXaTop) {
        const int d = top - kXaTop - a.e;
        xa_sra(a.hi, a.lo, d);
        a.e += d;
    }
    int s = e - a.e;  // <= kXaTop - len
    unsigned long long th, tl;
    if (s >= 0) {
        if (s >= 64) {
            th = pl << (s - 64);
            tl = 0;
        } else if (s > 0) {
            th = (ph << s) | (pl >> (64 - s));
            tl = pl << s;
        } else {
            th = ph;
            tl = pl;
        }
    } else {
        s = -s;
        if (s >= 128) {
            th = tl = 0;
        } else if (s >= 64) {
            tl = ph >> (s - 64);
            th = 0;
        } else {
            tl = (pl >> s) | (ph << (64 - s));
            th = ph >> s;
        }
    }
    if (neg) {
        tl = ~tl + 1ull;
        th = ~th + (tl == 0 ? 1ull : 0ull);
    }
    xa_add128(a.hi, a.lo, th, tl);
    xa_norm(a);
}

// x * y for FP64 operands.
__host__ __device__ __forceinline__ void xa_fma64(XAcc& a, double x, double y) {
#ifdef __CUDA_ARCH__
    const unsigned long long bx = (unsigned long long)__double_as_longlong(x);
    const unsigned long long by = (unsigned long long)__double_as_longlong(y);
#else
    unsigned long long bx, by;
    __builtin_memcpy(&bx, &x, 8);
    __builtin_memcpy(&by, &y, 8);
#endif
    const int Ex = (int)((bx >> 52) & 0x7FF), Ey = (int)((by >> 52) & 0x7FF);
    if (Ex == 0x7FF || Ey == 0x7FF) {
        a.e = kXaNaN;
        return;
    }
    unsigned long long mx = bx & 0xFFFFFFFFFFFFFull, my = by & 0xFFFFFFFFFFFFFull;
    if (Ex) mx |= 1ull << 52;
    if (Ey) my |= 1ull << 52;
    if (mx == 0 || my == 0) return;
    const int e = (Ex ? Ex - 1075 : -1074) + (Ey ? Ey - 1075 : -1074);
    xa_add_term(a, xa_mulhi64(mx, my), mx * my, e, ((bx ^ by) >> 63) != 0);
}

// x * y for FP32 operands (the product is at most 48 bits).
__host__ __device__ __forceinline__ void xa_fma32(XAcc& a, float x, float y) {
#ifdef __CUDA_ARCH__
    const unsigned bx = __float_as_uint(x), by = __float_as_uint(y);
#else
    unsigned bx, by;
    __builtin_memcpy(&bx, &x, 4);
    __builtin_memcpy(&by, &y, 4);
#endif
    const int Ex = (int)((bx >> 23) & 0xFF), Ey = (int)((by >> 23) & 0xFF);
    if (Ex == 0xFF || Ey == 0xFF) {
        a.e = kXaNaN;
        return;
    }
    unsigned mx = bx & 0x7FFFFFu, my = by & 0x7FFFFFu;
    if (Ex) mx |= 1u << 23;
    if (Ey) my |= 1u << 23;
    if (mx == 0 || my == 0) return;
    const int e = (Ex ? Ex - 150 : -149) + (Ey ? Ey - 150 : -149);
    xa_add_term(a, 0ull, (unsigned long long)mx * my, e, ((bx ^ by) >> 31) != 0);
}

__host__ __device__ __forceinline__ void xa_acc(XAcc& a, double x, double y) { xa_fma64(a, x, y); }
__host__ __device__ __forceinline__ void xa_acc(XAcc& a, float x, float y) { xa_fma32(a, x, y); }

// a += b (both exact accumulators); symmetric, so both partners of a
// butterfly step obtain bitwise the same result.
__host__ __device__ __forceinline__ void xa_merge(XAcc& a, const XAcc& b) {
    if (a.e == kXaNaN || b.e == kXaNaN) {
        a.e = kXaNaN;
        return;
    }
    if (b.e == kXaEmpty) return;
    if (a.e == kXaEmpty) {
        a = b;
        return;
    }
    const int E = a.e > b.e ? a.e : b.e;
    unsigned long long ah = a.hi, al = a.lo, bh = b.hi, bl = b.lo;
    xa_sra(ah, al, E - a.e);
    xa_sra(bh, bl, E - b.e);
    xa_add128(ah, al, bh, bl);
    a.hi = ah;
    a.lo = al;
    a.e = E;
    xa_norm(a);
}

// Round w * 2^e to the nearest FP64 (ties to even).
__host__ __device__ __forceinline__ double xa_round(const XAcc& a) {
    if (a.e == kXaEmpty) return 0.0;
    unsigned long long bits;
    if (a.e == kXaNaN) {
        bits = 0x7FF8000000000000ull;
    } else {
        unsigned long long hi = a.hi, lo = a.lo;
        const bool neg = (long long)hi < 0;
        if (neg) {
            lo = ~lo + 1ull;
            hi = ~hi + (lo == 0 ? 1ull : 0ull);
        }
        const int len = hi ? 128 - xa_clz64(hi) : 64 - xa_clz64(lo);
        if (len == 0) return 0.0;
        int q = a.e + len - 53;  // weight of the last kept bit
        if (q < -1074) q = -1074;
        const int sh = q - a.e;  // bits dropped
        unsigned long long mant;
        if (sh <= 0) {
            mant = lo << (-sh);  // len <= 53 here: exact
        } else {
            unsigned long long mh = hi, ml = lo;
            unsigned long long rh = hi, rl = lo;
            xa_sra(mh, ml, sh);  // value is non-negative here, so arithmetic == logical
            mant = ml;
            // round bit and sticky bits below the kept part
            xa_sra(rh, rl, sh - 1);
            const bool rbit = (rl & 1ull) != 0;
            bool sticky;
            const int sb = sh - 1;  // number of bits below the round bit
            if (sb <= 0) {
                sticky = false;
            } else if (sb >= 128) {
                sticky = (hi | lo) != 0;
            } else if (sb >= 64) {
                sticky = lo != 0 || (hi & ((sb == 64) ? 0ull : ((1ull << (sb - 64)) - 1ull))) != 0;
            } else {
                sticky = (lo & ((1ull << sb) - 1ull)) != 0;
            }
            if (rbit && (sticky || (mant & 1ull))) mant += 1ull;
        }
        if (mant >> 53) {
            mant >>= 1;
            q += 1;
        }
        if (mant >> 52) {
            const int E = q + 1075;
            bits = E >= 2047 ? (0x7FFull << 52) : (((unsigned long long)E << 52) | (mant & 0xFFFFFFFFFFFFFull));
        } else {
            bits = mant;  // subnormal (q == -1074)
        }
        if (neg) bits |= 1ull << 63;
    }
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)bits);
#else
    double r;
    __builtin_memcpy(&r, &bits, 8);
    return r;
#endif
}

#ifdef __CUDACC__
__device__ __forceinline__ XAcc xa_shfl_xor(const XAcc& a, int off) {
    XAcc b;
    b.e = __shfl_xor_sync(0xffffffffu, a.e, off);
    b.hi = __shfl_xor_sync(0xffffffffu, a.hi, off);
    b.lo = __shfl_xor_sync(0xffffffffu, a.lo, off);
    return b;
}
__device__ __forceinline__ void xa_warp_merge(XAcc& a) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const XAcc b = xa_shfl_xor(a, off);
        xa_merge(a, b);
    }
}
#endif

}  // namespace bcs
