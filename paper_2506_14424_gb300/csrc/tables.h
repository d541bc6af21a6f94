#pragma once
#include "common.cuh"

namespace sipg {
void gauss_legendre(int n, double* x, double* w);
void gauss_lobatto(int n, double* x, double* w);
Tab make_tab(int n);
SplitTab make_split_tab(int n);
TransferTab make_p_transfer(int nf, int nc);
TransferTab make_h_transfer(int n);
TransferTab make_p_interp_down(int nf, int nc);
TransferTab make_h_interp_down(int n, int* child);
LoadTab make_load_tab(int n);
}  // namespace sipg
