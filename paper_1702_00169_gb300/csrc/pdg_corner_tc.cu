// Instantiations of the tensor-core corner kernel (pdg_corner_tc.cuh) for degrees 1-3 and
// both residual precisions, its shared-memory size, and the host-side layout of its
// Binv operands.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>

#include "pdg_corner_tc.cuh"

namespace {

template <int NP>
size_t tc_smem(const PdgCornerPass& p) {
  return pdgdev::TcSmem<NP>(p.tx + p.c.wx, p.ty + p.c.wy, p.tz + p.c.wz, p.tc_layers == 2 ? 2 : 1).total;
}

template <int NP, int RES>
int go(const PdgCornerPass& p, size_t smem, cudaStream_t st) {
  auto kern = p.tc_layers == 2 ? pdgdev::corner_tc_kernel<NP, RES, 2> : pdgdev::corner_tc_kernel<NP, RES, 1>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  const long long blocks = (long long)p.ntx * p.nty * p.ntz * p.npop;
  kern<<<(unsigned)blocks, pdgdev::TcShape<NP>::THREADS, smem, st>>>(p);
  return (int)cudaGetLastError();
}

float tf32_round_host(float x) {
  // round to 10 explicit mantissa bits, to nearest, ties away (the device's cvt.rna.tf32)
  uint32_t b;
  std::memcpy(&b, &x, 4);
  if ((b & 0x7f800000u) != 0x7f800000u) b = (b + 0x1000u) & 0xffffe000u;
  float r;
  std::memcpy(&r, &b, 4);
  return r;
}

}  // namespace

size_t pdg_corner_tc_smem(const PdgCornerPass& p) {
  switch (p.n) {
    case 2: return tc_smem<2>(p);
    case 3: return tc_smem<3>(p);
    case 4: return tc_smem<4>(p);
  }
  return 0;
}

int pdg_launch_corner_tc(const PdgCornerPass& p, size_t smem, void* stream) {
  const long long blocks = (long long)p.ntx * p.nty * p.ntz * p.npop;
  if (blocks > 0x7fffffffLL || blocks < 1) return (int)cudaErrorInvalidConfiguration;
  const int layers = p.tc_layers == 2 ? 2 : 1;
  if (layers * std::min(p.tx + p.c.wx, p.ty + p.c.wy) > 128 || !p.binv_tc || !p.err) return (int)cudaErrorInvalidValue;
  cudaStream_t st = (cudaStream_t)stream;
  const int res = p.tc == 2 ? 1 : 0;
  switch (p.n * 2 + res) {
    case 4: return go<2, 0>(p, smem, st);
    case 5: return go<2, 1>(p, smem, st);
    case 6: return go<3, 0>(p, smem, st);
    case 7: return go<3, 1>(p, smem, st);
    case 8: return go<4, 0>(p, smem, st);
    case 9: return go<4, 1>(p, smem, st);
  }
  return (int)cudaErrorInvalidValue;
}

int pdg_corner_tc_operands(int n, const double* binv, float* out) {
  const int NN = n * n * n, K = (NN + 7) & ~7, N = K < 16 ? 16 : K;
  for (int i = 0; i < 2 * N * K; ++i) out[i] = 0.0f;
  for (int q = 0; q < NN; ++q)        // output node: the MMA's N index
    for (int m = 0; m < NN; ++m) {    // input node: the contraction index
      const double v = binv[q * NN + m];
      const float hi = tf32_round_host((float)v);
      const float lo = tf32_round_host((float)(v - (double)hi));
      const int idx = pdgdev::tc::op_index(q, m, N);
      out[idx] = hi;
      out[N * K + idx] = lo;
    }
  return 2 * N * K;
}
