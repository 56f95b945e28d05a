// Instantiation of the three-way ACA kernels for the Galerkin single layer
// (4 x 4-point rule); the kernel and its device routines live in
// g3_aca_dev.cuh, the host driver in g3_aca.cu.
#include "g3_aca_dev.cuh"

namespace g3 {

#define G3_ACA_INST(T, NT, DENSE)                                                                    \
    template g3_status launch_aca_t<G3_GAL_SLP, T, NT, DENSE>(g3_ctx*, AcaArgs<T>&, int, size_t);        \
    template int occupancy<G3_GAL_SLP, T, NT, DENSE>(size_t);

G3_ACA_INST(float, 256, false)
G3_ACA_INST(float, 256, true)
G3_ACA_INST(float, 512, false)
G3_ACA_INST(double, 256, false)
G3_ACA_INST(double, 256, true)

}  // namespace g3
