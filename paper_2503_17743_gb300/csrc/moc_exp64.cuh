// FP64 attenuation factor e^{-x} for the double-precision sweep (Eq. 3).
//
// Written from P. T. P. Tang, "Table-driven implementation of the exponential
// function in IEEE floating-point arithmetic", ACM TOMS 15(2), 1989: with
// n = round(-x 64 / ln 2), n = 64 m + j (0 <= j < 64) and r = -x - n ln2/64,
//     e^{-x} = 2^m * 2^{j/64} * e^r,   |r| <= ln2/128.
// 2^{j/64} is a table of hi + lo doubles (hi the nearest double, lo the
// nearest double to the remainder); ln2/64 = kStepHi + kStepLo with kStepHi
// holding 29 significant bits so that n * kStepHi is exact for |n| < 2^24;
// e^r - 1 = r + r^2 (1/2! + r/3! + r^2/4! + r^3/5!), the Taylor series cut
// after r^5 (dropped terms below r^6/6! < 3.6e-17 relative).  The result is
// hi + (lo + hi (e^r - 1)); the exponent m goes straight into the high word.
//
// Domain: |x| < 700 (the sweep's optical lengths Sigma_t l are >= 0), where
// the result is a normal double within about 0.7 ulp of e^{-x}; x >= 700 gives
// 0 (e^{-700} < 1e-304), x <= -700 +inf, NaN gives NaN.  Eleven FP64 operations, two
// integer tests and one 16-byte shared-memory load: the FP64 pipe is the
// bound of the double-precision sweep on this part.
#pragma once

#include <cstdint>

namespace moc_exp64 {

constexpr double kInvStep = 0x1.71547652b82fep+6;  // 64 / ln 2
constexpr double kStepHi = 0x1.62e42fe000000p-7;   // ln2/64, leading 29 bits
constexpr double kStepLo = 0x1.f473de6af278fp-36;  // ln2/64 - kStepHi
constexpr double kShift = 0x1.8p+52;               // 1.5 * 2^52: x + kShift rounds x to an integer in the low word
constexpr int kHiCut = 0x4085E000;                 // high word of 700.0
constexpr double kC2 = 0x1.0000000000000p-1;       // 1/2!
constexpr double kC3 = 0x1.5555555555555p-3;       // 1/3!
constexpr double kC4 = 0x1.5555555555555p-5;       // 1/4!
constexpr double kC5 = 0x1.1111111111111p-7;       // 1/5!

// 2^{j/64} = hi + lo, j = 0..63 (constant memory in CUDA translation units;
// the sweep copies it to shared memory once per block)
struct Pow2 {
    double hi, lo;
};
#ifdef __CUDACC__
#define MOC_EXP64_SPACE __constant__
#else
#define MOC_EXP64_SPACE
#endif
static MOC_EXP64_SPACE const Pow2 kTable[64] = {
    {0x1.0000000000000p+0, 0.0},
    {0x1.02c9a3e778061p+0, -0x1.19083535b085dp-56},
    {0x1.059b0d3158574p+0, 0x1.d73e2a475b465p-55},
    {0x1.0874518759bc8p+0, 0x1.186be4bb284ffp-57},
    {0x1.0b5586cf9890fp+0, 0x1.8a62e4adc610bp-54},
    {0x1.0e3ec32d3d1a2p+0, 0x1.03a1727c57b53p-59},
    {0x1.11301d0125b51p+0, -0x1.6c51039449b3ap-54},
    {0x1.1429aaea92de0p+0, -0x1.32fbf9af1369ep-54},
    {0x1.172b83c7d517bp+0, -0x1.19041b9d78a76p-55},
    {0x1.1a35beb6fcb75p+0, 0x1.e5b4c7b4968e4p-55},
    {0x1.1d4873168b9aap+0, 0x1.e016e00a2643cp-54},
    {0x1.2063b88628cd6p+0, 0x1.dc775814a8495p-55},
    {0x1.2387a6e756238p+0, 0x1.9b07eb6c70573p-54},
    {0x1.26b4565e27cddp+0, 0x1.2bd339940e9d9p-55},
    {0x1.29e9df51fdee1p+0, 0x1.612e8afad1255p-55},
    {0x1.2d285a6e4030bp+0, 0x1.0024754db41d5p-54},
    {0x1.306fe0a31b715p+0, 0x1.6f46ad23182e4p-55},
    {0x1.33c08b26416ffp+0, 0x1.32721843659a6p-54},
    {0x1.371a7373aa9cbp+0, -0x1.63aeabf42eae2p-54},
    {0x1.3a7db34e59ff7p+0, -0x1.5e436d661f5e3p-56},
    {0x1.3dea64c123422p+0, 0x1.ada0911f09ebcp-55},
    {0x1.4160a21f72e2ap+0, -0x1.ef3691c309278p-58},
    {0x1.44e086061892dp+0, 0x1.89b7a04ef80d0p-59},
    {0x1.486a2b5c13cd0p+0, 0x1.3c1a3b69062f0p-56},
    {0x1.4bfdad5362a27p+0, 0x1.d4397afec42e2p-56},
    {0x1.4f9b2769d2ca7p+0, -0x1.4b309d25957e3p-54},
    {0x1.5342b569d4f82p+0, -0x1.07abe1db13cadp-55},
    {0x1.56f4736b527dap+0, 0x1.9bb2c011d93adp-54},
    {0x1.5ab07dd485429p+0, 0x1.6324c054647adp-54},
    {0x1.5e76f15ad2148p+0, 0x1.ba6f93080e65ep-54},
    {0x1.6247eb03a5585p+0, -0x1.383c17e40b497p-54},
    {0x1.6623882552225p+0, -0x1.bb60987591c34p-54},
    {0x1.6a09e667f3bcdp+0, -0x1.bdd3413b26456p-54},
    {0x1.6dfb23c651a2fp+0, -0x1.bbe3a683c88abp-57},
    {0x1.71f75e8ec5f74p+0, -0x1.16e4786887a99p-55},
    {0x1.75feb564267c9p+0, -0x1.0245957316dd3p-54},
    {0x1.7a11473eb0187p+0, -0x1.41577ee04992fp-55},
    {0x1.7e2f336cf4e62p+0, 0x1.05d02ba15797ep-56},
    {0x1.82589994cce13p+0, -0x1.d4c1dd41532d8p-54},
    {0x1.868d99b4492edp+0, -0x1.fc6f89bd4f6bap-54},
    {0x1.8ace5422aa0dbp+0, 0x1.6e9f156864b27p-54},
    {0x1.8f1ae99157736p+0, 0x1.5cc13a2e3976cp-55},
    {0x1.93737b0cdc5e5p+0, -0x1.75fc781b57ebcp-57},
    {0x1.97d829fde4e50p+0, -0x1.d185b7c1b85d1p-54},
    {0x1.9c49182a3f090p+0, 0x1.c7c46b071f2bep-56},
    {0x1.a0c667b5de565p+0, -0x1.359495d1cd533p-54},
    {0x1.a5503b23e255dp+0, -0x1.d2f6edb8d41e1p-54},
    {0x1.a9e6b5579fdbfp+0, 0x1.0fac90ef7fd31p-54},
    {0x1.ae89f995ad3adp+0, 0x1.7a1cd345dcc81p-54},
    {0x1.b33a2b84f15fbp+0, -0x1.2805e3084d708p-57},
    {0x1.b7f76f2fb5e47p+0, -0x1.5584f7e54ac3bp-56},
    {0x1.bcc1e904bc1d2p+0, 0x1.23dd07a2d9e84p-55},
    {0x1.c199bdd85529cp+0, 0x1.11065895048ddp-55},
    {0x1.c67f12e57d14bp+0, 0x1.2884dff483cadp-54},
    {0x1.cb720dcef9069p+0, 0x1.503cbd1e949dbp-56},
    {0x1.d072d4a07897cp+0, -0x1.cbc3743797a9cp-54},
    {0x1.d5818dcfba487p+0, 0x1.2ed02d75b3707p-55},
    {0x1.da9e603db3285p+0, 0x1.c2300696db532p-54},
    {0x1.dfc97337b9b5fp+0, -0x1.1a5cd4f184b5cp-54},
    {0x1.e502ee78b3ff6p+0, 0x1.39e8980a9cc8fp-55},
    {0x1.ea4afa2a490dap+0, -0x1.e9c23179c2893p-54},
    {0x1.efa1bee615a27p+0, 0x1.dc7f486a4b6b0p-54},
    {0x1.f50765b6e4540p+0, 0x1.9d3e12dd8a18bp-54},
    {0x1.fa7c1819e90d8p+0, 0x1.74853f3a5931ep-55},
};

#ifdef __CUDACC__
// the table staged in shared memory by the calling block (64 x 16 bytes)
__device__ __forceinline__ double exp_neg(double x, const double2 *tab) {
    const double t = fma(x, -kInvStep, kShift);
    const int n = __double2loint(t);
    const double nd = t - kShift;
    double r = fma(nd, -kStepHi, -x);
    r = fma(nd, -kStepLo, r);
    const double r2 = r * r;
    double q = fma(kC5, r, kC4);
    q = fma(q, r, kC3);
    q = fma(q, r, kC2);
    const double pm1 = fma(q, r2, r);
    const double2 T = tab[n & 63];
    const double s = fma(T.x, pm1, T.y) + T.x;
    const double y = __hiloint2double(__double2hiint(s) + ((n >> 6) << 20), __double2loint(s));
    const int hx = __double2hiint(x), ax = hx & 0x7FFFFFFF;
    if (ax < kHiCut) return y;
    // |x| >= 700 or NaN: NaN passed through, 0 for x >= 700, +inf for x <= -700
    const bool nan = ax > 0x7FF00000 || (ax == 0x7FF00000 && __double2loint(x) != 0);
    return nan ? x : (hx < 0 ? __longlong_as_double(0x7FF0000000000000LL) : 0.0);
}
#endif

}  // namespace moc_exp64
