// Double-precision instantiation of the propagation kernels.
#include "tsbz_kernels.cuh"

template void launch_field<double>(const LaunchSet&, int, void*);
template void launch_bra<double>(const LaunchSet&, const void*, void*, int, int, void*);
template void launch_stage<double>(const LaunchSet&, const void*, void*, void*, const void*, int, void*);
template void launch_observe<double>(const LaunchSet&, const void*, double*, double*, double*, void*);
template void launch_finalize_t<double>(const SubDev*, int, const UnitDev*, const CellDev*, const double*,
                                        const void*, const double*, const double*, const double*, const int*, int,
                                        int, void*);
template int launch_hxc_t<double>(const SubDev*, const int*, int, const CellDev&, double2*, double2*,
                                  double2* const[3], void*);
template void launch_convert_in_t<double>(const double2*, void*, long long, void*);
template void launch_convert_out_t<double>(const void*, double2*, long long, void*);
template void launch_veff_frozen_t<double>(const SubDev*, int, const CellDev&, void*);
template void launch_veff_keep_t<double>(const SubDev*, const CellDev*, int, int, void*);
