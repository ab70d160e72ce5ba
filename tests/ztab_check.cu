// Host check of the Z-term tables (qv_device.cuh, ztab_build): for Z strings of
// every shape (the identity, chains inside and across 8-bit chunks, wide random
// masks), the tables plus the terms they leave give the same coefficient
// sum_k c_k (-1)^popcount(i & z_k) as the terms one by one, at random indices.
// Host code only: nothing runs on a GPU.
#include <cmath>
#include <cstdio>
#include <random>
#include <vector>

#include "qv_device.cuh"

int main()
{
    std::mt19937_64 rng(7);
    long bad = 0;
    for (int n : {5, 8, 12, 17, 20, 27, 33, 40}) {
        const uint64_t mask = (uint64_t(1) << n) - 1;
        std::vector<uint64_t> z = {0};
        std::vector<double> cr = {0.75}, ci = {0.0};
        for (int i = 0; i + 1 < n; ++i) {
            z.push_back((uint64_t(1) << i) | (uint64_t(1) << (i + 1)));
            cr.push_back(1.0 - 0.01 * i);
            ci.push_back(0.0);
        }
        for (int k = 0; k < 8; ++k) {
            z.push_back(rng() & mask);
            cr.push_back(0.1 * (k + 1));
            ci.push_back(0.05 * (k + 1));
        }
        const int nt = int(z.size());
        std::vector<uint64_t> z2 = z;
        std::vector<double> cr2 = cr, ci2 = ci, tab(qv::kZTabWords);
        int nch = 0;
        const int keep = qv::ztab_build(n, z2.data(), cr2.data(), ci2.data(), nt, tab.data(), &nch);
        for (int s = 0; s < 4000; ++s) {
            const uint64_t i = rng() & mask;
            double wr = 0, wi = 0, gr = 0, gi = 0;
            for (int k = 0; k < nt; ++k) {
                const double sg = (__builtin_popcountll(i & z[k]) & 1) ? -1.0 : 1.0;
                wr += sg * cr[k];
                wi += sg * ci[k];
            }
            for (int c = 0; c < nch; ++c) {
                const unsigned v = unsigned(i >> (8 * c)) & 255u;
                gr += tab[c * 256 + v];
                gi += tab[(qv::kZChunks + c) * 256 + v];
            }
            for (int k = 0; k < keep; ++k) {
                const double sg = (__builtin_popcountll(i & z2[k]) & 1) ? -1.0 : 1.0;
                gr += sg * cr2[k];
                gi += sg * ci2[k];
            }
            if (std::fabs(gr - wr) > 1e-12 || std::fabs(gi - wi) > 1e-12) ++bad;
        }
        std::printf("n %d chunks %d tabled %d of %d\n", n, nch, nt - keep, nt);
    }
    std::printf("bad %ld\n", bad);
    return bad != 0;
}
