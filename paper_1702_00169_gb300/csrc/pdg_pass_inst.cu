// Explicit instantiations of the pass kernels (pdg_pass_kernels.cuh) for one group of
// model variants and one number type, selected at compile time:
//   PDG_INST_T      0 = FP64, 1 = double-float;
//   PDG_INST_GROUP  0 = no collision, advection, shallow water, 1-D Euler;
//                   1 = 2-D and 3-D Euler;  2 = D2Q9, D3Q19;  3 = D3Q15, D3Q27.
// build.py compiles this file once per (type, group), in parallel.
#include "pdg_pass_kernels.cuh"

#if !defined(PDG_INST_T) || !defined(PDG_INST_GROUP)
#error "PDG_INST_T and PDG_INST_GROUP must be defined"
#endif

namespace pdgdev {
#if PDG_INST_T == 0
#define PDG_T double
#else
#define PDG_T dd
#endif
#define PDG_INST(MV) template int launch_pass_mv<MV, PDG_T>(const PdgPass&, cudaStream_t);
#if PDG_INST_GROUP == 0
PDG_INST(MV_NONE)
PDG_INST(MV_ADV)
PDG_INST(MV_SW)
PDG_INST(MV_EU1)
#elif PDG_INST_GROUP == 1
PDG_INST(MV_EU2)
PDG_INST(MV_EU3)
#elif PDG_INST_GROUP == 2
PDG_INST(MV_D2Q9)
PDG_INST(MV_D3Q19)
#elif PDG_INST_GROUP == 3
PDG_INST(MV_D3Q15)
PDG_INST(MV_D3Q27)
#endif
}  // namespace pdgdev
