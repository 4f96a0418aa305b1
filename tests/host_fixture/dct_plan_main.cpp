// Prints the DCT plan's FFT stage order for each length L given on the
// command line: "L ok r0 r1 ..." (ok 0 if L is not 13-smooth).  Host code
// only: links the library and calls its planner.
#include <cstdint>
#include <cstdio>
#include <cstdlib>

namespace sk {
bool dct_factor(int64_t L, int *fac, int *nf);
}

int main(int argc, char **argv) {
    for (int a = 1; a < argc; ++a) {
        const int64_t L = std::atoll(argv[a]);
        int fac[16], nf = 0;
        const bool ok = sk::dct_factor(L, fac, &nf);
        std::printf("%lld %d", (long long)L, ok ? 1 : 0);
        for (int q = 0; ok && q < nf; ++q) std::printf(" %d", fac[q]);
        std::printf("\n");
    }
    return 0;
}
