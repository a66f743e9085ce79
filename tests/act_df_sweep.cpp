// Host build of the FP64 activation's double-float arithmetic (csrc/act_df.cuh, the
// same FP32 operations as on the device, no contraction) swept against extended
// precision. Prints: max |z - z_ref|, max relative error of s and t, the count of
// non-finite outputs, and the special-value checks (1 = pass).
#include <cmath>
#include <cstdio>
#include <random>

#include "../paper_2510_00884_gb300/csrc/act_df.cuh"

using commet::actdf::f2;
static f2 tab[commet::actdf::kSlots];
static double zabs = 0, srel = 0, trel = 0;
static long nonfinite = 0;

static void check(double y) {
    double z, s, t;
    commet::actdf::softplus3(y, z, s, t, tab);
    if (!std::isfinite(z) || !std::isfinite(s) || !std::isfinite(t)) ++nonfinite;
    long double ay = std::fabs((long double)y);
    if (ay > 700.0L) ay = 700.0L;
    const long double e = std::exp(-ay);
    const long double w = 1.0L / (1.0L + e);
    const long double zr = (y > 0 ? (long double)y : 0.0L) + std::log1p(e);
    const long double sr = std::signbit(y) ? e * w : w;
    const long double tr = e * w * w;
    zabs = std::fmax(zabs, (double)std::fabs(z - zr));
    srel = std::fmax(srel, (double)(std::fabs(s - sr) / sr));
    trel = std::fmax(trel, (double)(std::fabs(t - tr) / tr));
}

int main(int argc, char **argv) {
    const long n = argc > 1 ? std::atol(argv[1]) : 1000000;
    commet::actdf::make_table(tab);
    std::mt19937_64 g(20251001);
    std::uniform_real_distribution<double> U(-1.0, 1.0);
    for (long i = 0; i < n; ++i) check(12.0 * U(g));
    for (long i = 0; i < n / 4; ++i) check(120.0 * U(g));
    for (long i = 0; i < n / 8; ++i) check(1e-3 * U(g));
    for (long i = 0; i < n / 8; ++i) check(800.0 * U(g));
    // both sides of every log-table cell edge, e = (k + 1/2)/256, and of the regime edge
    for (int k = 0; k < 256; ++k) {
        const double y = -std::log((k + 0.5) / 256.0);
        for (int d = -20; d <= 20; ++d) {
            check(y * (1.0 + d * 1e-15));
            check(-y * (1.0 + d * 1e-15));
        }
    }
    for (double y : {0.0, -0.0, 1e-300, -1e-300, 41.58, -41.58, 41.59, -41.59, 700.0, -700.0, 1e10, -1e10})
        check(y);
    double z, s, t;
    commet::actdf::softplus3(0.0, z, s, t, tab);
    const int zero_ok = std::fabs(z - std::log(2.0)) < 1e-15 && s == 0.5 && t == 0.25;
    commet::actdf::softplus3(50.0, z, s, t, tab);
    const int big_ok = z == 50.0 && s == 1.0 && std::fabs(t / std::exp(-50.0) - 1.0) < 1e-14;
    commet::actdf::softplus3(-50.0, z, s, t, tab);
    const int small_ok = std::fabs(z / std::exp(-50.0) - 1.0) < 1e-14 && s == z && t == z;
    std::printf("%.6e %.6e %.6e %ld %d %d %d\n", zabs, srel, trel, nonfinite, zero_ok, big_ok, small_ok);
    return 0;
}
