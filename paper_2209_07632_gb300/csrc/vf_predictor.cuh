// The rank predictor's inference, for assembly (vf_predictor.cu).
#pragma once

#include <vector>

#include "vf_internal.cuh"

namespace vf {

// Classes (argmax, ties to the lower class) and probabilities (n x
// VF_PRED_NCLASS) of n feature rows (n x VF_PRED_NFEAT, host).
vf_status predictor_classify(const vf_rank_predictor* p, const std::vector<float>& feats, int64_t n,
                             std::vector<int32_t>& cls, std::vector<float>& prob);

}  // namespace vf
