// tlog.cuh -- the natural logarithm of the FP64 lubrication term.
//
// Table-driven method of P. T. P. Tang (ACM Trans. Math. Softw. 16(4),
// 1990): x = 2^k m with m in [1, 2); F_j = 1 + j/128 is the table point
// nearest m (j from the leading eight bits of the mantissa, rounded), so
// f = m - F_j is exact and |f| <= 1/256; u = f / F_j (f times the tabulated
// 1/F_j), and
//   ln x = (k ln2_hi + hi_j) + (ln(1 + u) + (k ln2_lo + lo_j)),
// where the first sum is exact (both terms are multiples of 2^-42) and
// ln(1 + u) is its Taylor series to u^7 (the next term is below 2^-67).  The
// error stays below one unit in the last place plus 2^-60.  Every product and
// sum is spelled out with round-to-nearest operations, so the host and the
// device compile it to the same results; the host build is what the tests
// check against high-precision values.  It needs about half the FP64
// instructions of the library logarithm, the largest single item of the FP64
// pair kernel.  Arguments that are not positive normal finite numbers go to
// log().
#pragma once
#include <cmath>
#include <cstring>

#include "log_table.cuh"

namespace dps {

static __device__ const double tlog_table_dev[129][4] = {DPS_LOG_TABLE_ROWS};
static const double tlog_table_host[129][4] = {DPS_LOG_TABLE_ROWS};

__host__ __device__ __forceinline__ double tl_fma(double a, double b, double c) {
#ifdef __CUDA_ARCH__
    return __fma_rn(a, b, c);
#else
    return std::fma(a, b, c);
#endif
}
__host__ __device__ __forceinline__ double tl_mul(double a, double b) {
#ifdef __CUDA_ARCH__
    return __dmul_rn(a, b);
#else
    return a * b;
#endif
}
__host__ __device__ __forceinline__ double tl_add(double a, double b) {
#ifdef __CUDA_ARCH__
    return __dadd_rn(a, b);
#else
    return a + b;
#endif
}
__host__ __device__ __forceinline__ double tl_sub(double a, double b) {
#ifdef __CUDA_ARCH__
    return __dsub_rn(a, b);
#else
    return a - b;
#endif
}

__host__ __device__ inline double tlog(double x) {
    if (!(x >= 0x1p-1022 && x <= 0x1.fffffffffffffp+1023)) return log(x);
    unsigned long long b;
    double m;
#ifdef __CUDA_ARCH__
    b = (unsigned long long)__double_as_longlong(x);
    const double(*T)[4] = tlog_table_dev;
#else
    std::memcpy(&b, &x, sizeof b);
    const double(*T)[4] = tlog_table_host;
#endif
    const int k = (int)(b >> 52) - 1023;               // x > 0: the sign bit is clear
    const int j = (int)((((b >> 44) & 0xffu) + 1u) >> 1);  // nearest 1/128: 0..128
    const unsigned long long mb = (b & 0x000fffffffffffffull) | 0x3ff0000000000000ull;
#ifdef __CUDA_ARCH__
    m = __longlong_as_double((long long)mb);
#else
    std::memcpy(&m, &mb, sizeof m);
#endif
    const double f = tl_sub(m, T[j][0]);
    const double u = tl_mul(f, T[j][1]);
    // ln(1 + u) = u + u^2 P(u), P(u) = -1/2 + u/3 - u^2/4 + u^3/5 - u^4/6 + u^5/7
    double p = tl_fma(1.0 / 7.0, u, -1.0 / 6.0);
    p = tl_fma(p, u, 1.0 / 5.0);
    p = tl_fma(p, u, -0.25);
    p = tl_fma(p, u, 1.0 / 3.0);
    p = tl_fma(p, u, -0.5);
    const double r = tl_fma(tl_mul(u, u), p, u);
    const double kd = (double)k;
    const double s = tl_fma(kd, DPS_LN2_HI, T[j][2]);  // exact
    const double t = tl_add(r, tl_fma(kd, DPS_LN2_LO, T[j][3]));
    return tl_add(s, t);
}

}  // namespace dps
