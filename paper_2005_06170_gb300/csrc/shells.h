// Host-side shell tables of the binning (plain C++, no CUDA): which |k| shell each
// integer |n|^2 belongs to, the shells as integer intervals of |n|^2, and the list of
// (slab, shell) work items that hold modes. Built once per context and grid size by
// build_spectra_tables; compiled into the library and, on its own, into a CPU test.
#ifndef PKMOM_SHELLS_H
#define PKMOM_SHELLS_H

#include <cstdint>
#include <vector>

namespace pkmom {

// Linear shells of u = |n| (|k| in units of the fundamental frequency) on [umin, umax],
// nbins of them: bintab[nsq] is the shell of |n|^2 = nsq (0xFFFF outside the range; the
// same FP64 expression as the definition of the bins), thresh[b] <= |n|^2 < thresh[b+1]
// is shell b (nbins + 1 entries; shells are monotone in |n|^2, an empty shell has
// thresh[b] == thresh[b+1]). Returns nsq_max, the largest |n|^2 the table covers.
int shell_tables(int nbins, double umin, double umax, std::vector<uint16_t> &bintab, std::vector<int> &thresh);

// The (slab, shell) items i0 * nbins + b of an ng^3 half spectrum in which shell b
// reaches slab n_x = n0 (thresh[b+1] - 1 >= n0^2), slabs by increasing |n0| (0, -1, 1,
// -2, ...) and the outer shells of a slab first. Items missing from the list hold no
// mode.
std::vector<uint32_t> bin_item_list(const std::vector<int> &thresh, int ng, int nbins);

}  // namespace pkmom

#endif
