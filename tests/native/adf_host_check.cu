// Host check of the aligned double-float arithmetic of the FFT lines
// (csrc/adf.cuh, compiled here for the CPU): Stockham transforms built from
// its butterflies, in the stage schedule of the GPU lines, against a direct
// long-double DFT of the same input.
//
//   pow2 mode: the register-resident plans (radix 8, then 2 or 4), the grid
//     chosen from the line's bound with 2^19 headroom, 16x coarser per stage;
//   mixed mode: {2,3,5}-smooth plans, first stage exact (the GPU runs it in
//     double-float), then aligned stages on the grid of that stage's bound
//     with 2^18 headroom and the generic growth R sqrt(2) per stage.
//
// Prints one line per (plan, input pattern): the largest error over
// L * (input bound), and the largest |hi| / q seen at a stage input, as
// log2 (the grid invariant: <= 19, resp. 18).
#include <cmath>
#include <cstdio>
#include <random>
#include <vector>

#include "adf.cuh"
using namespace mvd;

static cdd mk(long double re, long double im) {
    const float rh = (float)re, ih = (float)im;
    return cdd{dd{rh, (float)(re - rh)}, dd{ih, (float)(im - ih)}};
}

template <int S>
static void bfly(int R, cdd* v, float c) {
    switch (R) {
        case 8: DftA<8, S>::run(v, c); break;
        case 4: DftA<4, S>::run(v, c); break;
        case 2: DftA<2, S>::run(v, c); break;
        case 3: DftA<3, S>::run(v, c); break;
        case 5: DftA<5, S>::run(v, c); break;
        case 6: DftA<6, S>::run(v, c); break;
        case 9: DftA<9, S>::run(v, c); break;
    }
}

static int gap_of(const cdd& v, int e) {
    const float m = fmaxf(fabsf(v.re.hi), fabsf(v.im.hi));
    return m > 0.f ? (int)std::ceil(std::log2((double)m) - e) : -1000;
}

// forward transform (S = -1) of x in place; returns the largest grid gap
static int fft_aligned(std::vector<cdd>& x, const std::vector<int>& plan, bool pow2) {
    const int L = (int)x.size();
    std::vector<cdd> tw(L), B(L);
    for (int m = 0; m < L; ++m) {
        const long double a = -2.0L * M_PIl * m / L;
        tw[m] = mk(cosl(a), sinl(a));
    }
    int e = 0, gap = -1000, Ns = 1;
    float c = 0.f, M = 0.f;
    if (pow2) {
        for (auto& v : x) M = adf_absmax(v, M);
        e = adf_exp_for(M);
        c = adf_const_exp2(e);
        for (auto& v : x) v = adf_calign(v, c);
    }
    for (size_t s = 0; s < plan.size(); ++s) {
        const int R = plan[s];
        if (pow2 && s > 0) e += adf_stage_shift(plan[s - 1]);
        if (!pow2 && s == 1) e = adf_exp_for<18>(1.5f * M);
        if (!pow2 && s > 1) e += adf_gen_shift(plan[s - 1]);
        c = adf_const_exp2(e);
        for (int j = 0; j < L / R; ++j) {
            const int k = j % Ns;
            cdd v[9];
            for (int r = 0; r < R; ++r) v[r] = x[j + r * (L / R)];
            if (!pow2 && s == 0) {  // the exact first stage
                long double yr[9], yi[9];
                for (int m = 0; m < R; ++m) {
                    long double sr = 0, si = 0;
                    for (int r = 0; r < R; ++r) {
                        const long double a = -2.0L * M_PIl * ((r * m) % R) / R;
                        const long double xr = (long double)v[r].re.hi + v[r].re.lo;
                        const long double xi = (long double)v[r].im.hi + v[r].im.lo;
                        sr += xr * cosl(a) - xi * sinl(a);
                        si += xr * sinl(a) + xi * cosl(a);
                    }
                    yr[m] = sr;
                    yi[m] = si;
                }
                for (int m = 0; m < R; ++m) {
                    v[m] = mk(yr[m], yi[m]);
                    M = adf_absmax(v[m], M);
                }
            } else {
                if (Ns > 1) {
                    const int step = k * (L / (Ns * R));
                    v[0] = adf_calign(v[0], c);
                    for (int r = 1; r < R; ++r) v[r] = adf_cmul(v[r], tw[r * step], c);
                }
                for (int r = 0; r < R; ++r) {
                    const int g = gap_of(v[r], e);
                    if (g > gap) gap = g;
                }
                bfly<-1>(R, v, c);
            }
            const int d = (j / Ns) * Ns * R + k;
            for (int r = 0; r < R; ++r) B[d + r * Ns] = v[r];
        }
        x.swap(B);
        Ns *= R;
    }
    return gap;
}

int main(int argc, char** argv) {
    const bool pow2 = argc > 1 && argv[1][0] == 'p';
    std::vector<std::vector<int>> plans;
    if (pow2)
        plans = {{8, 4}, {8, 8}, {8, 8, 2}, {8, 8, 4}, {8, 8, 8}, {8, 8, 8, 2}};
    else
        plans = {{4, 4, 3, 5}, {3, 3, 3, 3, 3}, {5, 5, 3}, {9, 4, 4}, {6, 6, 6}, {8, 9, 3},
                 {5, 4, 4, 4}, {9, 9, 2}, {8, 8, 5}, {6, 5, 3, 3}, {2, 2, 2, 3}};
    std::mt19937_64 g(7);
    std::uniform_real_distribution<double> U(0, 1);
    for (const auto& p : plans) {
        int L = 1;
        for (int r : p) L *= r;
        for (int pat = 0; pat < 7; ++pat) {
            std::vector<cdd> x(L);
            for (int n = 0; n < L; ++n) {
                long double re = 0, im = 0;
                switch (pat) {
                    case 0: re = U(g); im = U(g); break;                                   // uniform
                    case 1: re = 3.7; im = -1.1; break;                                   // constant
                    case 2: re = U(g) < 0.01 ? 1e6 * U(g) : 1e-3 * U(g); break;           // spikes
                    case 3:                                                               // 8 decades
                        re = powl(10.0L, -8 * U(g)) * (U(g) - .5);
                        im = powl(10.0L, -8 * U(g)) * (U(g) - .5);
                        break;
                    case 4: re = (n & 1) ? -1 : 1; im = -re; break;                       // alternating
                    case 5: re = cosl(2 * M_PIl * 7 * n / L); im = sinl(2 * M_PIl * 7 * n / L); break;
                    default: re = U(g) * 1e3 + U(g) * 1e-5; im = U(g) * 1e-4; break;      // low parts
                }
                x[n] = mk(re, im);
            }
            std::vector<long double> xr(L), xi(L);
            long double inmax = 0;
            for (int n = 0; n < L; ++n) {
                xr[n] = (long double)x[n].re.hi + x[n].re.lo;
                xi[n] = (long double)x[n].im.hi + x[n].im.lo;
                inmax = fmaxl(inmax, fmaxl(fabsl(xr[n]), fabsl(xi[n])));
            }
            const int gap = fft_aligned(x, p, pow2);
            long double emax = 0;
            for (int k = 0; k < L; ++k) {
                long double sr = 0, si = 0;
                for (int n = 0; n < L; ++n) {
                    const long double a = -2.0L * M_PIl * (long double)((long)n * k % L) / L;
                    sr += xr[n] * cosl(a) - xi[n] * sinl(a);
                    si += xr[n] * sinl(a) + xi[n] * cosl(a);
                }
                emax = fmaxl(emax, fmaxl(fabsl((long double)x[k].re.hi + x[k].re.lo - sr),
                                         fabsl((long double)x[k].im.hi + x[k].im.lo - si)));
            }
            printf("%d %d %.6Le %d\n", L, pat, emax / (inmax * L), gap);
        }
    }
    return 0;
}
