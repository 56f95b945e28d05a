// Instantiation of the three-way ACA kernels for the single-layer kernel; the kernel and its
// device routines live in g3_aca_dev.cuh, the host driver in g3_aca.cu.
#include "g3_aca_dev.cuh"

namespace g3 {

#define G3_ACA_INST(T, NT, DENSE)                                                                    \
    template g3_status launch_aca_t<G3_SLP, T, NT, DENSE>(g3_ctx*, AcaArgs<T>&, int, size_t);        \
    template int occupancy<G3_SLP, T, NT, DENSE>(size_t);

// compiled in four parts (G3_ACA_PART = 0, 1, 2, 3) by separate compiler processes
#if !defined(G3_ACA_PART) || G3_ACA_PART == 0
G3_ACA_INST(float, 256, false)
G3_ACA_INST(float, 128, false)
#endif
#if !defined(G3_ACA_PART) || G3_ACA_PART == 1
G3_ACA_INST(float, 256, true)
G3_ACA_INST(float, 512, false)
#endif
#if !defined(G3_ACA_PART) || G3_ACA_PART == 2
G3_ACA_INST(double, 256, false)
G3_ACA_INST(double, 256, true)
#endif
#if !defined(G3_ACA_PART) || G3_ACA_PART == 3
G3_ACA_INST(float, 384, false)
template g3_status launch_whole_t<G3_SLP, float>(g3_ctx*, AcaArgs<float>&, int, size_t, int, int, const double*,
                                               WholeCand*, Cx<double>*, double*);
template g3_status launch_whole_fiber_t<G3_SLP, float>(g3_ctx*, AcaArgs<float>&, int, int, int, int, Cx<double>*,
                                                     Cx<double>*, double*, int, const Cx<double>*, const double*,
                                                     double*, double*);
#endif
#if !defined(G3_ACA_PART) || G3_ACA_PART == 2
template g3_status launch_whole_t<G3_SLP, double>(g3_ctx*, AcaArgs<double>&, int, size_t, int, int, const double*,
                                                WholeCand*, Cx<double>*, double*);
template g3_status launch_whole_fiber_t<G3_SLP, double>(g3_ctx*, AcaArgs<double>&, int, int, int, int, Cx<double>*,
                                                      Cx<double>*, double*, int, const Cx<double>*, const double*,
                                                      double*, double*);
#endif

}  // namespace g3
