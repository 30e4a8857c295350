// hodlr.cu -- HODLR compression and application (placeholder until the kernels land).
#include "hodlr.cuh"
#include "kernels.cuh"

namespace ddst {

void HodlrSet::clear() { release(); }

void HodlrSet::release() {
  for (void* p : {UV, D, (void*)t, (void*)acc, (void*)d_blocks, (void*)d_leaves})
    if (p) cudaFree(p);
  UV = D = nullptr;
  t = acc = nullptr;
  d_blocks = nullptr;
  d_leaves = nullptr;
  blocks.clear();
  leaves.clear();
  built = false;
  bytes = 0;
  max_rank = 0;
}

template <typename T>
int hodlr_build(HodlrSet& H, const HodlrParams&, const std::vector<SlabDesc>&,
                const std::vector<ProbDesc>&, const SlabDesc*, const T*, cudaStream_t,
                std::string& msg) {
  H.release();
  msg = "HODLR compression not available";
  return 1;
}

template <typename T>
void hodlr_apply(HodlrSet&, const SlabDesc*, const ProbDesc*, int, const double*, double*, int,
                 cudaStream_t) {}

int hodlr_expand(HodlrSet&, int, int, size_t, double*, cudaStream_t) { return 1; }

template int hodlr_build<float>(HodlrSet&, const HodlrParams&, const std::vector<SlabDesc>&,
                                const std::vector<ProbDesc>&, const SlabDesc*, const float*,
                                cudaStream_t, std::string&);
template int hodlr_build<double>(HodlrSet&, const HodlrParams&, const std::vector<SlabDesc>&,
                                 const std::vector<ProbDesc>&, const SlabDesc*, const double*,
                                 cudaStream_t, std::string&);
template void hodlr_apply<float>(HodlrSet&, const SlabDesc*, const ProbDesc*, int, const double*,
                                 double*, int, cudaStream_t);
template void hodlr_apply<double>(HodlrSet&, const SlabDesc*, const ProbDesc*, int, const double*,
                                  double*, int, cudaStream_t);

}  // namespace ddst
