// Host harness for the solver's 3 x 3 eigen-step (small_sym_eig_min, rayleigh_ritz of
// csrc/lane_update.cuh, the Rayleigh-Ritz step of the LOBPCG iteration for lambda_min of
// Lemma 3.1).  Both functions are __host__ __device__; this program runs their host form on
// cases read from stdin, one per line, and prints one result line per case:
//   eig k m00 m01 m02 m11 m12 m22      ->  lam v0 v1 v2
//   rr has_p ga0 .. ga5 gb0 .. gb5     ->  ok lam c0 c1 c2   |   fail
// Test infrastructure only (tests/test_eigenstep_host.py builds and runs it).
#include <cstdio>
#include <cstring>

#include "../paper_2408_04875_gb300/csrc/lane_update.cuh"

int main()
{
    char kind[8];
    while (std::scanf("%7s", kind) == 1) {
        if (std::strcmp(kind, "eig") == 0) {
            int k;
            float a[6];
            if (std::scanf("%d %f %f %f %f %f %f", &k, &a[0], &a[1], &a[2], &a[3], &a[4], &a[5]) != 7) return 2;
            float M[3][3] = {{a[0], a[1], a[2]}, {a[1], a[3], a[4]}, {a[2], a[4], a[5]}};
            float lam, v[3];
            ubqp::small_sym_eig_min(k, M, lam, v);
            std::printf("%.9g %.9g %.9g %.9g\n", lam, v[0], v[1], v[2]);
        } else if (std::strcmp(kind, "rr") == 0) {
            int has_p;
            float ga[6], gb[6];
            if (std::scanf("%d", &has_p) != 1) return 2;
            for (int t = 0; t < 6; ++t)
                if (std::scanf("%f", &ga[t]) != 1) return 2;
            for (int t = 0; t < 6; ++t)
                if (std::scanf("%f", &gb[t]) != 1) return 2;
            float lam = 0.f, c[3] = {0.f, 0.f, 0.f};
            if (ubqp::rayleigh_ritz(ga, gb, has_p != 0, lam, c))
                std::printf("ok %.9g %.9g %.9g %.9g\n", lam, c[0], c[1], c[2]);
            else
                std::printf("fail\n");
        } else {
            return 2;
        }
    }
    return 0;
}
