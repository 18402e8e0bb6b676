// Host-side table builders (tsbz_host.cpp).
#pragma once
#include <vector>

#include "tsbz.h"

namespace tsbz {
void fd_weights(int nd, double* c, double* d);
void local_potential(const tsbz_cell_desc& d, std::vector<double>& out);
void projector_tables(const tsbz_cell_desc& d, std::vector<double>& g1, std::vector<double>& d1,
                      std::vector<double>& pnorm, int nmax);
}  // namespace tsbz
