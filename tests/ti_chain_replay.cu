// Host replay of the thermodynamic-integration chains (Algorithm 3) with the library's own
// per-chain arithmetic (ti.cuh, compiled here for the host): the sequence of ti_start, ti_init,
// T x ti_step and ti_finish, with the per-X-string sums S(a) read from a table instead of the
// per-X kernels.  Used by tests/test_ti_chain_host.py to compare the chains with the oracle's.
//
// usage: ti_chain_replay S.bin N L n_s burn_in seed eps even out.bin
// out.bin: int32 nonpos flag, (L + 3) doubles (means, I, M_2, delta M_2), L * T int64 trajectory.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "ti.cuh"

using namespace hm;

int main(int argc, char** argv) {
    if (argc != 10) return 2;
    const int N = atoi(argv[2]), L = atoi(argv[3]);
    const long long n_s = atoll(argv[4]), burn = atoll(argv[5]);
    const unsigned long long seed = strtoull(argv[6], nullptr, 10);
    const double eps = atof(argv[7]);
    const int even = atoi(argv[8]);
    std::vector<double> S((size_t)1 << N);
    FILE* f = fopen(argv[1], "rb");
    if (!f || fread(S.data(), sizeof(double), S.size(), f) != S.size()) return 3;
    fclose(f);
    const long long T = burn + n_s;
    std::vector<long long> a(L), prop(L), traj((size_t)L * T);
    const int B = ti_n_batches(n_s);
    const long long K = n_s / B;
    std::vector<double> fe(L), acc(L), out(L + 3), bsum((size_t)L * B, 0.0);
    int nonpos = 0;
    auto energy = [&](double s) {
        const double x = s + eps;
        if (!(x > 0.0)) nonpos = 1;
        return -log(x);
    };
    for (int l = 0; l < L; ++l) {  // ti_start
        a[l] = ti_start_pattern(seed, l, N, even);
        prop[l] = a[l];
    }
    for (int l = 0; l < L; ++l) {  // ti_init
        fe[l] = energy(S[prop[l]]);
        acc[l] = 0.0;
        prop[l] = a[l] ^ ti_move(seed, l, 0, N, even);
    }
    for (long long t = 0; t < T; ++t)  // ti_step
        for (int l = 0; l < L; ++l) {
            const double f2 = energy(S[prop[l]]);
            double fa = fe[l];
            long long x = a[l];
            if (ti_accept(ti_uniform(seed, l, t), ti_beta(l, L), f2, fa)) {
                x = prop[l];
                fa = f2;
                a[l] = x;
                fe[l] = fa;
            }
            if (t >= burn) {
                acc[l] += fa;
                const long long b = (t - burn) / K;
                if (b < B) bsum[(size_t)l * B + b] += fa;
            }
            traj[(size_t)l * T + t] = x;
            if (t + 1 < T) prop[l] = x ^ ti_move(seed, l, t + 1, N, even);
        }
    double I = 0.0, var_I = 0.0;  // ti_finish
    for (int l = 0; l < L; ++l) {
        const double w = ti_simpson_weight(l, L);
        out[l] = acc[l] / (double)n_s;
        I += w * out[l];
        var_I += w * w * ti_chain_var(bsum.data() + (size_t)l * B, B, K);
    }
    out[L] = I;
    out[L + 1] = ti_m2(I, eps, even);
    out[L + 2] = B < 2 ? 0.0 : ti_m2_slope(I, eps) * sqrt(var_I);
    FILE* o = fopen(argv[9], "wb");
    if (!o) return 4;
    fwrite(&nonpos, sizeof(int), 1, o);
    fwrite(out.data(), sizeof(double), out.size(), o);
    fwrite(traj.data(), sizeof(long long), traj.size(), o);
    fclose(o);
    return 0;
}
