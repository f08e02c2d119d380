// Double-word FP32 arithmetic (a value is the unevaluated sum h + l of two floats),
// built from the error-free transformations TwoSum (Knuth) and TwoProduct via FMA
// as analysed in Joldes, Muller, Popescu, "Tight and rigorous error bounds for
// basic building blocks of double-word arithmetic", ACM TOMS 44 (2017).
// Accumulators are kept unnormalised (h + l) and normalised before storage;
// accuracy is a few units of 2^-48 relative to the magnitudes involved.
#pragma once
#include "common.cuh"

namespace ddamg {

struct dw {
    float h, l;
};

__device__ __forceinline__ dw two_sum(float a, float b) {
    float s = a + b;
    float bb = s - a;
    float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}

// acc += x * y  (x double-word, y double-word; acc kept unnormalised: h + l)
__device__ __forceinline__ void dw_mac(dw& acc, dw x, dw y) {
    float p = x.h * y.h;
    float e = fmaf(x.h, y.h, -p);
    e = fmaf(x.h, y.l, e);
    e = fmaf(x.l, y.h, e);
    dw s = two_sum(acc.h, p);
    acc.h = s.h;
    acc.l = acc.l + (s.l + e);
}
// acc += x * y for a float y
__device__ __forceinline__ void dw_macf(dw& acc, dw x, float y) {
    float p = x.h * y;
    float e = fmaf(x.h, y, -p);
    e = fmaf(x.l, y, e);
    dw s = two_sum(acc.h, p);
    acc.h = s.h;
    acc.l = acc.l + (s.l + e);
}
__device__ __forceinline__ dw dw_neg(dw a) { return {-a.h, -a.l}; }
__device__ __forceinline__ dw dw_add(dw a, dw b) {
    dw s = two_sum(a.h, b.h);
    s.l += a.l + b.l;
    return s;
}
__device__ __forceinline__ dw dw_norm(dw a) {
    float s = a.h + a.l;
    return {s, a.l - (s - a.h)};
}

struct cdw {
    dw re, im;
};
__device__ __forceinline__ cdw cdw_zero() { return {{0.f, 0.f}, {0.f, 0.f}}; }
// acc += b * c
__device__ __forceinline__ void cdw_mac(cdw& acc, const cdw& b, const cdw& c) {
    dw_mac(acc.re, b.re, c.re);
    dw_mac(acc.re, dw_neg(b.im), c.im);
    dw_mac(acc.im, b.re, c.im);
    dw_mac(acc.im, b.im, c.re);
}
// acc += conj(b) * c
__device__ __forceinline__ void cdw_mac_conj(cdw& acc, const cdw& b, const cdw& c) {
    dw_mac(acc.re, b.re, c.re);
    dw_mac(acc.re, b.im, c.im);
    dw_mac(acc.im, b.re, c.im);
    dw_mac(acc.im, dw_neg(b.im), c.re);
}
template <int P>
__device__ __forceinline__ cdw cdw_ipow(const cdw& a) {
    if (P == 0) return a;
    if (P == 1) return {dw_neg(a.im), a.re};
    if (P == 2) return {dw_neg(a.re), dw_neg(a.im)};
    return {a.im, dw_neg(a.re)};
}
__device__ __forceinline__ cdw cdw_add(const cdw& a, const cdw& b) { return {dw_add(a.re, b.re), dw_add(a.im, b.im)}; }
__device__ __forceinline__ cdw cdw_sub(const cdw& a, const cdw& b) { return {dw_add(a.re, dw_neg(b.re)), dw_add(a.im, dw_neg(b.im))}; }

__device__ __forceinline__ cdw cdw_zero_() { return {{0.f, 0.f}, {0.f, 0.f}}; }
__device__ __forceinline__ dw dw_from_double(double x) {
    float h = (float)x;
    return {h, (float)(x - (double)h)};
}
__device__ __forceinline__ double dw_to_double(dw a) { return (double)a.h + (double)a.l; }
__device__ __forceinline__ dw fast_two_sum(float a, float b) {
    float s = a + b;
    return {s, b - (s - a)};
}

}  // namespace ddamg
