// Host-side shell tables of the binning (see shells.h). No device code: the file is
// compiled by nvcc into the library and by a plain C++ compiler into a CPU test.
#include "shells.h"

#include <algorithm>
#include <cmath>

namespace pkmom {

int shell_tables(int nbins, double umin, double umax, std::vector<uint16_t> &bintab, std::vector<int> &thresh)
{
    const int nsq_max = static_cast<int>(std::floor(umax * umax)) + 1;
    bintab.assign(nsq_max + 1, 0xffff);
    for (int nsq = 1; nsq <= nsq_max; ++nsq) {
        const double u = std::sqrt(static_cast<double>(nsq));
        if (u < umin || u > umax) continue;
        double tb = std::floor(((u - umin) * nbins) / (umax - umin));
        if (tb > nbins - 1) tb = nbins - 1;
        bintab[nsq] = static_cast<uint16_t>(tb);
    }
    // shell b is the interval thresh[b] <= |n|^2 < thresh[b + 1] (bins are monotone in |n|^2)
    thresh.assign(nbins + 1, nsq_max + 1);
    int last = 0;
    for (int nsq = nsq_max; nsq >= 1; --nsq) {
        const int b = bintab[nsq];
        if (b == 0xffff) continue;
        if (!last) last = nsq;
        for (int k = b; k >= 0 && thresh[k] > nsq; --k) thresh[k] = nsq;
    }
    thresh[nbins] = last + 1;
    for (int k = nbins - 1; k >= 0; --k) thresh[k] = std::min(thresh[k], thresh[k + 1]);
    return nsq_max;
}

std::vector<uint32_t> bin_item_list(const std::vector<int> &thresh, int ng, int nbins)
{
    std::vector<uint32_t> work;
    for (int r = 0; r < ng; ++r) {
        const int k = r >> 1, i0 = (r & 1) ? ng - 1 - k : k;
        const int n0 = i0 < ng / 2 ? i0 : i0 - ng;
        for (int b = nbins - 1; b >= 0; --b)
            if (thresh[b + 1] > thresh[b] && thresh[b + 1] - 1 - n0 * n0 >= 0)
                work.push_back(static_cast<uint32_t>(i0) * nbins + b);
    }
    return work;
}

}  // namespace pkmom
