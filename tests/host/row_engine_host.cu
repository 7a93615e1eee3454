// Host-side checks of the row engine's compile-time parts (built by
// tests/test_host_row_engine.py with nvcc, run on the CPU):
//   "plan M VALS TPR THREADS NPASS R0 R1 R2"  RowPlan<M> for every row length
//   "dft R err"  the largest deviation of the in-register R-point DFTs
//                (forward and inverse, with and without the zero-input and
//                half-output forms) from a direct double-precision DFT of the
//                same float inputs.
#include <cmath>
#include <cstdio>
#include <cstdlib>

#include "graf_fft.cuh"

using namespace graf;

template <int M>
void plan() {
    using P = RowPlan<M>;
    std::printf("plan %d %d %d %d %d %d %d %d\n", M, P::VALS, P::TPR, P::THREADS, P::NPASS, P::R0, P::R1, P::R2);
}

template <int R, bool INV, bool HIN, bool HOUT>
double dft_err() {
    float2 v[R];
    double xr[R], xi[R];
    for (int i = 0; i < R; ++i) {
        const bool zero = HIN && i >= R / 2;
        xr[i] = zero ? 0.0 : (float)(std::rand() / (double)RAND_MAX - 0.5);
        xi[i] = zero ? 0.0 : (float)(std::rand() / (double)RAND_MAX - 0.5);
        v[i] = make_float2((float)xr[i], (float)xi[i]);
    }
    dft<R, 0, 1, INV, HIN, HOUT>(v);
    double err = 0.0;
    for (int k = 0; k < (HOUT ? R / 2 : R); ++k) {
        double ar = 0.0, ai = 0.0;
        for (int n = 0; n < R; ++n) {
            const double a = (INV ? 2.0 : -2.0) * M_PI * (double)((k * n) % R) / R;
            ar += xr[n] * std::cos(a) - xi[n] * std::sin(a);
            ai += xr[n] * std::sin(a) + xi[n] * std::cos(a);
        }
        err = std::fmax(err, std::fmax(std::fabs(ar - v[k].x), std::fabs(ai - v[k].y)));
    }
    return err;
}

template <int R>
void dft_all() {
    const double e[8] = {dft_err<R, false, false, false>(), dft_err<R, true, false, false>(),
                         dft_err<R, false, true, false>(),  dft_err<R, true, true, false>(),
                         dft_err<R, false, false, true>(),  dft_err<R, true, false, true>(),
                         dft_err<R, false, true, true>(),   dft_err<R, true, true, true>()};
    double m = 0.0;
    for (double x : e) m = std::fmax(m, x);
    std::printf("dft %d %.6e\n", R, m);
}

int main() {
    std::srand(2506);
    plan<8>(); plan<16>(); plan<32>(); plan<64>(); plan<128>(); plan<256>(); plan<512>();
    plan<1024>(); plan<2048>(); plan<4096>(); plan<8192>(); plan<16384>();
    dft_all<2>(); dft_all<4>(); dft_all<8>(); dft_all<16>(); dft_all<32>(); dft_all<64>();
    return 0;
}
