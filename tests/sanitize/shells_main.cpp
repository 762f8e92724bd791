// CPU check of the binning's host-side shell tables (paper_2005_06170_gb300/csrc/shells.cu)
// against brute force over every mode of small half spectra: each |n|^2 in exactly the
// shell interval its table entry names (and in none when outside the range), the
// intervals ordered, and the item list holding every (slab, shell) pair that has a mode,
// once, slabs by increasing |n0|.
#include <cstdio>
#include <cstdlib>
#include <set>
#include <vector>

#include "shells.h"

static int fails = 0;
#define CHECK(c, ...)                                  \
    do {                                               \
        if (!(c)) {                                    \
            std::printf("FAIL %s:%d ", __FILE__, __LINE__); \
            std::printf(__VA_ARGS__);                  \
            std::printf("\n");                         \
            ++fails;                                   \
        }                                              \
    } while (0)

static void one(int ng, int nbins, double umin, double umax)
{
    std::vector<uint16_t> bintab;
    std::vector<int> thresh;
    const int nsq_max = pkmom::shell_tables(nbins, umin, umax, bintab, thresh);
    CHECK(static_cast<int>(bintab.size()) == nsq_max + 1 && static_cast<int>(thresh.size()) == nbins + 1,
          "sizes ng=%d", ng);
    for (int b = 0; b < nbins; ++b) CHECK(thresh[b] <= thresh[b + 1], "order b=%d", b);
    for (int nsq = 1; nsq <= nsq_max; ++nsq) {
        int in = -1, count = 0;
        for (int b = 0; b < nbins; ++b)
            if (thresh[b] <= nsq && nsq < thresh[b + 1]) in = b, ++count;
        if (bintab[nsq] == 0xffff) CHECK(count == 0, "nsq=%d outside the range but in shell %d", nsq, in);
        else CHECK(count == 1 && in == bintab[nsq], "nsq=%d table %d intervals %d (%d)", nsq, bintab[nsq], in, count);
    }
    // brute force: the (slab, shell) items that hold at least one mode of the half spectrum
    std::set<uint32_t> held;
    const int nh = ng / 2 + 1;
    for (int i0 = 0; i0 < ng; ++i0)
        for (int i1 = 0; i1 < ng; ++i1)
            for (int l = 0; l < nh; ++l) {
                const int n0 = i0 < ng / 2 ? i0 : i0 - ng, n1 = i1 < ng / 2 ? i1 : i1 - ng;
                const int nsq = n0 * n0 + n1 * n1 + l * l;
                for (int b = 0; b < nbins; ++b)
                    if (thresh[b] <= nsq && nsq < thresh[b + 1]) held.insert(static_cast<uint32_t>(i0) * nbins + b);
            }
    const std::vector<uint32_t> work = pkmom::bin_item_list(thresh, ng, nbins);
    std::set<uint32_t> listed(work.begin(), work.end());
    CHECK(listed.size() == work.size(), "duplicates ng=%d", ng);
    for (uint32_t it : held) CHECK(listed.count(it) == 1, "item %u with modes not listed (ng=%d)", it, ng);
    int last_abs = -1;
    for (uint32_t it : work) {
        const int i0 = static_cast<int>(it) / nbins, b = static_cast<int>(it) % nbins;
        const int n0 = i0 < ng / 2 ? i0 : i0 - ng, a = n0 < 0 ? -n0 : n0;
        CHECK(i0 < ng && thresh[b + 1] - 1 >= n0 * n0, "listed item %u misses its slab", it);
        CHECK(a >= last_abs, "slab order |n0| %d after %d", a, last_abs);
        last_abs = a;
    }
    std::printf("ng=%d nbins=%d u=[%g, %g]: %zu items listed, %zu hold modes\n", ng, nbins, umin, umax, work.size(),
                held.size());
}

int main()
{
    one(16, 8, 1.0, 8.0);
    one(32, 16, 1.0, 16.0);
    one(24, 12, 1.0, 12.0);
    one(20, 7, 2.5, 9.3);
    one(16, 4, 0.5, 8.0);
    one(64, 128, 1.0, 32.0);  // more shells than integer radii: empty shells
    one(2, 1, 1.0, 1.0);
    if (fails) {
        std::printf("%d failures\n", fails);
        return 1;
    }
    std::printf("shells ok\n");
    return 0;
}
