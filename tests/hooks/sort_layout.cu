// Prints the radix sort's digit layout for every key width 0..32, one line
// per width: "<key_bits> <passes> <shift>:<bits> ..." (host code only; the
// device computes the same layout with the same function).
#include <cstdio>

#include "prims.cuh"

int main() {
    for (int kb = 0; kb <= 32; ++kb) {
        const int np = odp::prim::sort_passes(kb);
        std::printf("%d %d", kb, np);
        for (int p = 0; p < np + 2; ++p) {
            const odp::prim::SortPass sp = odp::prim::sort_pass(p, kb);
            if (sp.active) std::printf(" %d:%d", sp.shift, sp.bits);
            else std::printf(" -");
        }
        std::printf("\n");
    }
    return 0;
}
