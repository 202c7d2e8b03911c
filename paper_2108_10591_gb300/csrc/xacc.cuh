// Exact, order-independent inner-product accumulation on the integer pipes.
//
// Every product x_j y_j is formed exactly as an integer (53 x 53 -> 106 bits
// for FP64 operands, 24 x 24 -> 48 bits for FP32) with a power-of-two weight,
// and added into a 128-bit two's-complement fixed-point window
//     value = w * 2^e.
// The window is anchored so that the largest term seen so far fills its upper
// bits, with headroom above for the carries of the terms a lane adds; when a
// larger term arrives the window slides up.  Bits below the window's bottom
// (about 2^-107 of the warp's largest term, 2^-119 with the high placement of
// wa_acc) are dropped.  Partial accumulators from different threads and CTAs
// are aligned to the larger anchor and added as integers, and the final value
// is rounded once to FP64, nearest even.  The dropped bits add up to at most n
// times the bottom's weight, so the result is the correctly rounded inner
// product, independent of the order in which terms and partials were
// combined, unless the sum cancels below about n 2^-54 (n 2^-66) of its
// largest term.  No FP64 arithmetic is used, so the scarce FP64 units of the
// GPU stay with the recurrences and the SpMV.
#pragma once
#include <stdint.h>

namespace bcs {

constexpr int kXaTop = 110;              // anchor headroom: terms end at or below bit kXaTop
constexpr int kXaEmpty = -(1 << 29);     // e of an accumulator with no terms
constexpr int kXaNaN = (1 << 29);        // e of an accumulator that saw a NaN/Inf operand

// Merged partial sums (warp totals, CTA records, grid totals): 192-bit two's
// complement, value = (w2:w1:w0) * 2^e.  The per-lane partials of the solver
// use the cheaper 128-bit WAcc below; 192 bits leave room for every merge
// (at most 2^19 products per lane, 2^26 lanes) without dropping bits.
struct XAcc {
    int e;
    unsigned long long w2, w1, w0;
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
    a.w2 = a.w1 = a.w0 = 0;
}

// 128-bit helpers (per-lane partials)
__host__ __device__ __forceinline__ void xa_add128(unsigned long long& hi, unsigned long long& lo,
                                                   unsigned long long th, unsigned long long tl) {
    const unsigned long long l = lo + tl;
    hi = hi + th + (l < lo ? 1ull : 0ull);
    lo = l;
}

// 192-bit helpers: arithmetic shift right by d >= 0 (branch-free selects) and add.
__host__ __device__ __forceinline__ void xa_sar192(XAcc& a, int d) {
    const long long sg = (long long)a.w2 >> 63;
    unsigned long long w0 = a.w0, w1 = a.w1, w2 = a.w2;
    const int q = d >= 192 ? 3 : d / 64;   // whole words
    const int r = d >= 192 ? 0 : d % 64;   // bits
    // word shift
    const unsigned long long s2 = (unsigned long long)sg;
    unsigned long long t0 = q == 0 ? w0 : q == 1 ? w1 : q == 2 ? w2 : s2;
    unsigned long long t1 = q == 0 ? w1 : q == 1 ? w2 : s2;
    unsigned long long t2 = q == 0 ? w2 : s2;
    // bit shift
    if (r) {
        t0 = (t0 >> r) | (t1 << (64 - r));
        t1 = (t1 >> r) | (t2 << (64 - r));
        t2 = (unsigned long long)((long long)t2 >> r);
    }
    a.w0 = t0;
    a.w1 = t1;
    a.w2 = t2;
}
__host__ __device__ __forceinline__ void xa_add192(XAcc& a, unsigned long long b2, unsigned long long b1,
                                                   unsigned long long b0) {
    const unsigned long long s0 = a.w0 + b0;
    const unsigned long long c0 = s0 < a.w0 ? 1ull : 0ull;
    const unsigned long long s1a = a.w1 + b1;
    const unsigned long long c1a = s1a < a.w1 ? 1ull : 0ull;
    const unsigned long long s1 = s1a + c0;
    const unsigned long long c1 = c1a + (s1 < s1a ? 1ull : 0ull);
    a.w0 = s0;
    a.w1 = s1;
    a.w2 = a.w2 + b2 + c1;
}
// keep |w| < 2^188 (merges add at most a few bits before the next normalisation)
__host__ __device__ __forceinline__ void xa_norm(XAcc& a) {
    const long long t = (long long)a.w2 >> 60;
    if (t != 0 && t != -1) {
        xa_sar192(a, 8);
        a.e += 8;
    }
}

// a += b for two merged partials (general anchors); symmetric.
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
    XAcc x = a, y = b;
    xa_sar192(x, E - a.e);
    xa_sar192(y, E - b.e);
    xa_add192(x, y.w2, y.w1, y.w0);
    x.e = E;
    xa_norm(x);
    a = x;
}

// Round w * 2^e to the nearest FP64 (ties to even).
__host__ __device__ __forceinline__ double xa_round(const XAcc& a) {
    if (a.e == kXaEmpty) return 0.0;
    unsigned long long bits;
    if (a.e == kXaNaN) {
        bits = 0x7FF8000000000000ull;
    } else {
        unsigned long long w0 = a.w0, w1 = a.w1, w2 = a.w2;
        const bool neg = (long long)w2 < 0;
        if (neg) {  // negate
            w0 = ~w0;
            w1 = ~w1;
            w2 = ~w2;
            w0 += 1ull;
            const unsigned long long c0 = w0 == 0ull ? 1ull : 0ull;
            w1 += c0;
            w2 += (c0 && w1 == 0ull) ? 1ull : 0ull;
        }
        int len = w2 ? 192 - xa_clz64(w2) : w1 ? 128 - xa_clz64(w1) : 64 - xa_clz64(w0);
        if (len == 0) return 0.0;
        int q = a.e + len - 53;  // weight of the last kept bit
        if (q < -1074) q = -1074;
        const int sh = q - a.e;  // bits dropped
        unsigned long long mant;
        if (sh <= 0) {
            mant = w0 << (-sh);  // len <= 53 here: exact
        } else {
            XAcc m;
            m.e = 0;
            m.w0 = w0;
            m.w1 = w1;
            m.w2 = w2;  // non-negative: arithmetic == logical shift
            XAcc rb = m;
            xa_sar192(m, sh);
            mant = m.w0;
            xa_sar192(rb, sh - 1);
            const bool rbit = (rb.w0 & 1ull) != 0;
            // sticky: any of the lowest sh-1 bits
            const int sb = sh - 1;
            bool sticky;
            if (sb <= 0) sticky = false;
            else if (sb < 64) sticky = (w0 & ((1ull << sb) - 1ull)) != 0;
            else if (sb == 64) sticky = w0 != 0;
            else if (sb < 128) sticky = w0 != 0 || (w1 & ((1ull << (sb - 64)) - 1ull)) != 0;
            else if (sb == 128) sticky = (w0 | w1) != 0;
            else if (sb < 192) sticky = (w0 | w1) != 0 || (w2 & ((1ull << (sb - 128)) - 1ull)) != 0;
            else sticky = (w0 | w1 | w2) != 0;
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
// ---- per-warp accumulation with a warp-uniform window --------------------------------
//
// In the solver every lane adds one product per 32-row tile.  The 32 lanes of
// a warp share one window anchor: per term the warp takes the largest term
// top (five shuffles), slides the shared window up if needed (a uniform
// branch), and each lane then only shifts its term right into the window and
// adds it: no divergent branches, about 40 integer instructions per product.
constexpr int kWaTop = 108;        // the warp's largest term ends at or below bit kWaTop
constexpr int kWaNone = -(1 << 30);

struct WAcc {
    int eb;                        // exponent of bit 0 of the window; the same in all lanes of a warp
    unsigned long long hi, lo;     // this lane's 128-bit two's complement partial sum
};

__device__ __forceinline__ void wa_init(WAcc& a) {
    a.eb = kXaEmpty;
    a.hi = 0;
    a.lo = 0;
}

// (h:l) >>= r, logical, r >= 0, without branches (r >= 128 gives 0)
__device__ __forceinline__ void shr128(unsigned long long& h, unsigned long long& l, int r) {
    const int rr = r > 127 ? 127 : r;
    const int s = rr & 63;
    const unsigned long long lo_a = s ? ((l >> s) | (h << (64 - s))) : l;
    const unsigned long long hi_a = h >> s;
    const bool big = rr >= 64;
    l = big ? hi_a : lo_a;
    h = big ? 0ull : hi_a;
    if (r > 127) {
        h = 0ull;
        l = 0ull;
    }
}
// (h:l) >>= r, arithmetic, r >= 0, without branches
__device__ __forceinline__ void sar128(unsigned long long& h, unsigned long long& l, int r) {
    const long long sh = (long long)h;
    const int rr = r > 127 ? 127 : r;
    const int s = rr & 63;
    const unsigned long long lo_a = s ? ((l >> s) | (h << (64 - s))) : l;
    const unsigned long long hi_a = (unsigned long long)(sh >> s);
    const bool big = rr >= 64;
    l = big ? hi_a : lo_a;
    h = big ? (unsigned long long)(sh >> 63) : hi_a;
}

__device__ __forceinline__ int warp_max_int(int v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, off));
    return v;
}

// Add this lane's term (ph:pl) * 2^pe, where ph:pl < 2^kWaTop; `valid` lanes
// only; `special` marks a NaN/Inf operand.  Every lane of the warp must call.
__device__ __forceinline__ void wa_add_term(WAcc& a, unsigned long long ph, unsigned long long pl, int pe, bool neg,
                                            bool valid, bool special) {
    if (__any_sync(0xffffffffu, special)) a.eb = kXaNaN;
    if (a.eb == kXaNaN) return;
    const int top = valid ? pe + kWaTop : kWaNone;
    // the window moves only when some lane's term ends above it (one vote in
    // the common case; the warp maximum only when it has to move)
    if (!__all_sync(0xffffffffu, top <= a.eb + kWaTop)) {
        const int wmax = warp_max_int(top);
        if (a.eb == kXaEmpty) {
            a.eb = wmax - kWaTop;
        } else {
            const int d = wmax - kWaTop - a.eb;
            sar128(a.hi, a.lo, d);
            a.eb += d;
        }
    }
    shr128(ph, pl, a.eb - pe);
    if (!valid) {
        ph = 0ull;
        pl = 0ull;
    }
    if (neg) {
        pl = ~pl + 1ull;
        ph = ~ph + (pl == 0ull ? 1ull : 0ull);
    }
    xa_add128(a.hi, a.lo, ph, pl);
}

// x * y, FP64 operands: the exact 106-bit product shifted left by s (2 <= s <=
// 20), so that the warp's largest term fills bits up to 105 + s of the window
// and the window's bottom lies 105 + s bits below that term's top.  A lane adds
// k terms below 2^(106 + s), so its 128-bit sum cannot overflow while
// k <= 2^(21 - s); the solver picks the largest s its tiles per warp allow (the
// larger s, the fewer low bits of the smaller terms are dropped), s = 2 holds
// for up to 2^19 terms.
__device__ __forceinline__ void wa_acc(WAcc& a, double x, double y, bool valid, int s = 2) {
    const unsigned long long bx = (unsigned long long)__double_as_longlong(x);
    const unsigned long long by = (unsigned long long)__double_as_longlong(y);
    const int Ex = (int)((bx >> 52) & 0x7FF), Ey = (int)((by >> 52) & 0x7FF);
    const bool special = valid && (Ex == 0x7FF || Ey == 0x7FF);
    unsigned long long mx = (bx & 0xFFFFFFFFFFFFFull) | (Ex ? (1ull << 52) : 0ull);
    unsigned long long my = (by & 0xFFFFFFFFFFFFFull) | (Ey ? (1ull << 52) : 0ull);
    const bool live = valid && !special && mx != 0ull && my != 0ull;
    const unsigned long long ph = __umul64hi(mx, my), pl = mx * my;
    const int pe = (Ex ? Ex - 1075 : -1074) + (Ey ? Ey - 1075 : -1074) - s;
    wa_add_term(a, (ph << s) | (pl >> (64 - s)), pl << s, pe, ((bx ^ by) >> 63) != 0ull, live, special);
}

// x * y, FP32 operands: exact 48-bit product, placed with its top at bit 108.
__device__ __forceinline__ void wa_acc(WAcc& a, float x, float y, bool valid, int = 2) {
    const unsigned bx = __float_as_uint(x), by = __float_as_uint(y);
    const int Ex = (int)((bx >> 23) & 0xFF), Ey = (int)((by >> 23) & 0xFF);
    const bool special = valid && (Ex == 0xFF || Ey == 0xFF);
    const unsigned mx = (bx & 0x7FFFFFu) | (Ex ? (1u << 23) : 0u);
    const unsigned my = (by & 0x7FFFFFu) | (Ey ? (1u << 23) : 0u);
    const bool live = valid && !special && mx != 0u && my != 0u;
    const unsigned long long p = (unsigned long long)mx * my;
    const int pe = (Ex ? Ex - 150 : -149) + (Ey ? Ey - 150 : -149) - 60;
    wa_add_term(a, p >> 4, p << 60, pe, ((bx ^ by) >> 31) != 0u, live, special);
}

// Warp total of a WAcc: every lane obtains the exact warp sum as a 192-bit XAcc.
__device__ __forceinline__ XAcc wa_warp_total(const WAcc& a) {
    XAcc r;
    r.e = a.eb;
    r.w0 = a.lo;
    r.w1 = a.hi;
    r.w2 = (unsigned long long)((long long)a.hi >> 63);
    if (a.eb == kXaNaN || a.eb == kXaEmpty) {
        r.w0 = r.w1 = r.w2 = 0ull;
        return r;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long b0 = __shfl_xor_sync(0xffffffffu, r.w0, off);
        const unsigned long long b1 = __shfl_xor_sync(0xffffffffu, r.w1, off);
        const unsigned long long b2 = __shfl_xor_sync(0xffffffffu, r.w2, off);
        xa_add192(r, b2, b1, b0);
    }
    return r;
}

// Exact sum over the lanes of a warp of merged partials with different
// anchors, aligned to the largest anchor (bits below its window are dropped:
// more than 2^-108 below the largest product).  Every lane obtains the total.
__device__ __forceinline__ XAcc xa_warp_aligned_sum(XAcc a) {
    const int E = warp_max_int(a.e);
    XAcc r;
    r.e = E;
    r.w0 = r.w1 = r.w2 = 0ull;
    if (E == kXaNaN || E == kXaEmpty) return r;
    xa_sar192(a, E - a.e);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long b0 = __shfl_xor_sync(0xffffffffu, a.w0, off);
        const unsigned long long b1 = __shfl_xor_sync(0xffffffffu, a.w1, off);
        const unsigned long long b2 = __shfl_xor_sync(0xffffffffu, a.w2, off);
        xa_add192(a, b2, b1, b0);
    }
    a.e = E;
    xa_norm(a);
    return a;
}


// ---- FP64 per-lane accumulation (refinement modes: FP32 vectors) --------------------
// The inner products of the FP32 inner solves accumulate in FP64: each lane
// adds the exact product of its two FP32 operands (exact in FP64) with one
// FP64 fma; the lane sums are then merged exactly like the integer partials.
struct DAcc {
    double s;
};
__device__ __forceinline__ void wa_init(DAcc& a) { a.s = 0.0; }

// FP32 -> FP64 widening (exact).  The conversion instruction was measured
// faster than rebiasing the bits with integer operations (fewer issued
// instructions per tile).  A pure function of its operand, so the widening of
// a value that enters several inner products is computed once.
__device__ __forceinline__ double widen(float f) { return (double)f; }
__device__ __forceinline__ void wa_acc(DAcc& a, float x, float y, bool valid, int = 2) {
    if (valid) a.s = fma(widen(x), widen(y), a.s);
}

// exact 192-bit representation of a double, its significand placed at bits
// 70..122 so that aligning it to a partial up to 2^70 times larger keeps
// every bit (the merges then do not depend on how lanes are grouped)
constexpr int kXaDblShift = 70;
__device__ __forceinline__ XAcc xa_from_double(double d) {
    XAcc r;
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const int E = (int)((b >> 52) & 0x7FF);
    r.w2 = r.w1 = r.w0 = 0ull;
    if (E == 0x7FF) {
        r.e = kXaNaN;
        return r;
    }
    const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (E ? (1ull << 52) : 0ull);
    if (m == 0ull) {
        r.e = kXaEmpty;
        return r;
    }
    r.e = (E ? E - 1075 : -1074) - kXaDblShift;
    static_assert(kXaDblShift >= 64 && kXaDblShift + 53 <= 127, "significand inside w1");
    r.w1 = m << (kXaDblShift - 64);
    if (b >> 63) {  // negate
        r.w0 = ~r.w0;
        r.w1 = ~r.w1;
        r.w2 = ~0ull;
        r.w0 += 1ull;
        if (r.w0 == 0ull) {
            r.w1 += 1ull;
            if (r.w1 == 0ull) r.w2 += 1ull;
        }
    }
    return r;
}
__device__ __forceinline__ XAcc wa_warp_total(const DAcc& a) { return xa_warp_aligned_sum(xa_from_double(a.s)); }

// per-lane accumulator type of a solve: exact integer windows for FP64
// vectors, FP64 sums for FP32 vectors
template <class VT> struct DotAccOf { typedef WAcc type; };
template <> struct DotAccOf<float> { typedef DAcc type; };
#endif

}  // namespace bcs
