// FP64 instantiation of the batched persistent kernels and the dispatch by precision
// (see pdg_batch.cuh).
#include "pdg_batch.cuh"

int pdg_launch_batch_df(int np, int mv, const PdgPass* d_descs, const int* d_ent_desc,
                        const long long* d_ent_start, int nent, long long total, unsigned long long* d_counter,
                        size_t smem, void* stream);

int pdg_batch_threads() { return pdgdev::kBatchThreads; }

size_t pdg_batch_smem(int max_carry_doubles) {
  return sizeof(double) * ((size_t)pdgdev::kDescWords + (size_t)max_carry_doubles);
}

int pdg_launch_batch(const PdgPass* d_descs, const int* d_ent_desc, const long long* d_ent_start, int nent,
                     long long total, unsigned long long* d_counter, size_t smem, int prec, int np, int mv,
                     void* stream) {
  if (prec == PDG_PREC_DF32)
    return pdg_launch_batch_df(np, mv, d_descs, d_ent_desc, d_ent_start, nent, total, d_counter, smem, stream);
  return pdgdev::launch_batch_t<double>(np, mv, d_descs, d_ent_desc, d_ent_start, nent, total, d_counter, smem,
                                        stream);
}
