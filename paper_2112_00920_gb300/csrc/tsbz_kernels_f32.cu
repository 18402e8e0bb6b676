// Single-precision instantiation of the propagation kernels.
#include "tsbz_kernels.cuh"

template void launch_field<float>(const LaunchSet&, int, void*);
template void launch_bra<float>(const LaunchSet&, const void*, void*, int, int, void*);
template void launch_stage<float>(const LaunchSet&, const void*, void*, void*, const void*, int, void*);
template void launch_observe<float>(const LaunchSet&, const void*, double*, double*, double*, void*);
template void launch_finalize_t<float>(const SubDev*, int, const UnitDev*, const CellDev*, const double*,
                                        const void*, const double*, const double*, const double*, const int*, int,
                                        int, void*);
template int launch_hxc_t<float>(const SubDev*, const int*, int, const CellDev&, double2*, double2*,
                                  double2* const[3], void*);
template void launch_convert_in_t<float>(const double2*, void*, long long, void*);
template void launch_convert_out_t<float>(const void*, double2*, long long, void*);
template void launch_veff_frozen_t<float>(const SubDev*, int, const CellDev&, void*);
template void launch_veff_keep_t<float>(const SubDev*, const CellDev*, int, int, void*);
