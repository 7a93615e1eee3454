// Host-side dump of the launch configuration the library derives for a row
// length M (built by tests/test_host_launch_config.py with nvcc, run on the
// CPU):
//   "mirror M TPR THREADS SLOTS MIN_BLOCKS tpr_of threads_of slots_of"
//   "acc M N real per copies smem smem_2x"  gradient accumulators per CTA (0:
//        none fits), the backward kernel's shared memory with them (with one
//        if none fits) and with twice as many
//   "tile B M lo hi slots rows_per_tile tiles"
#include <cstdio>

#include "graf_kernels.cuh"

using namespace graf;

constexpr int kSms = 152;  // the SM count the tiling is checked with (a GB300)

template <int M>
void one() {
    using P = RowPlan<M>;
    constexpr int slots = P::THREADS / P::TPR;
    std::printf("mirror %d %d %d %d %d %d %d %d\n", M, P::TPR, P::THREADS, slots, P::MIN_BLOCKS, tpr_of(M),
                threads_of(M), slots_of(M));
    const int Ns[] = {1, M / 4 > 0 ? M / 4 : 1, M / 2, M / 2 + 1, M};
    for (int N : Ns) {
        for (int real = 0; real < 2; ++real) {
            for (int per = 0; per < (N == M ? 2 : 1); ++per) {
                const int a = backward_acc_copies<M>(N, real, per);
                // with no copy that fits (a = 0): the need of one copy
                const size_t s = backward_smem<M>(N, a ? a : 1, real, per);
                const size_t s2 = backward_smem<M>(N, a ? 2 * a : 2, real, per);
                std::printf("acc %d %d %d %d %d %zu %zu\n", M, N, real, per, a, s, s2);
            }
        }
    }
    const int Bs[] = {1, 7, 256, 4096};
    for (int B : Bs) {
        const int his[] = {0, 1, M / 2, M - 1};
        for (int hi : his) {
            if (hi < 0) continue;
            const Tiling T = make_tiling_rows(B, M, 0, hi, kSms);
            std::printf("tile %d %d %d %d %d %d %d\n", B, M, 0, hi, T.slots, T.rows_per_tile, T.tiles);
        }
    }
}

int main() {
    std::printf("const %zu %zu %d\n", kMaxSmem, kSmemPerSm, kSms);
    one<8>(); one<16>(); one<32>(); one<64>(); one<128>(); one<256>(); one<512>();
    one<1024>(); one<2048>(); one<4096>(); one<8192>(); one<16384>();
    return 0;
}
