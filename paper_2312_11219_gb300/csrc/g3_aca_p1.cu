// Instantiation of the three-way ACA kernels for the Galerkin operators of
// linear continuous elements (hypersingular operator, adjoint double layer) on
// element-local shape functions; the kernel and its device routines live in
// g3_aca_dev.cuh, the host driver in g3_aca.cu.  256 threads per CTA only.
#include "g3_aca_dev.cuh"

namespace g3 {

#define G3_ACA_INST(KER, T, NT, DENSE)                                                               \
    template g3_status launch_aca_t<KER, T, NT, DENSE>(g3_ctx*, AcaArgs<T>&, int, size_t);          \
    template int occupancy<KER, T, NT, DENSE>(size_t);

// compiled in four parts (G3_ACA_PART = 0, 1, 2, 3) by separate compiler processes
#if !defined(G3_ACA_PART) || G3_ACA_PART == 0
G3_ACA_INST(G3_GAL_P1D, float, 256, false)
G3_ACA_INST(G3_GAL_P1D, float, 256, true)
#endif
#if !defined(G3_ACA_PART) || G3_ACA_PART == 1
G3_ACA_INST(G3_GAL_P1KP, float, 256, false)
G3_ACA_INST(G3_GAL_P1KP, float, 256, true)
#endif
#if !defined(G3_ACA_PART) || G3_ACA_PART == 2
G3_ACA_INST(G3_GAL_P1D, double, 256, false)
G3_ACA_INST(G3_GAL_P1D, double, 256, true)
#endif
#if !defined(G3_ACA_PART) || G3_ACA_PART == 3
G3_ACA_INST(G3_GAL_P1KP, double, 256, false)
G3_ACA_INST(G3_GAL_P1KP, double, 256, true)
#endif

}  // namespace g3
