// Prints the P2 reference tables of the library (paper_2403_04491_gb300/csrc/p2_tables.cpp) for
// d = 2 and 3, one table per line: "<name> <d> <values...>" in row-major order.
#include <cstdio>

#include "p2_tables.h"

int main() {
    for (int d = 2; d <= 3; ++d) {
        const knp::P2Ref& R = knp::p2_ref(d);
        std::printf("mass %d", d);
        for (int j = 0; j < R.npe; ++j)
            for (int l = 0; l < R.npe; ++l) std::printf(" %.17g", R.mass[j][l]);
        std::printf("\nfmass %d", d);
        for (int j = 0; j < R.nfn; ++j)
            for (int l = 0; l < R.nfn; ++l) std::printf(" %.17g", R.fmass[j][l]);
        std::printf("\nftriple %d", d);
        for (int c = 0; c < R.nfn; ++c)
            for (int j = 0; j < R.nfn; ++j)
                for (int l = 0; l < R.nfn; ++l) std::printf(" %.17g", R.ftriple[c][j][l]);
        std::printf("\nnterms %d %d\n", d, R.nterms);
    }
    return 0;
}
