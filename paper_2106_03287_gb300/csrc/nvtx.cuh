// NVTX ranges around the library's calls and the method's stages, in the
// "steinicp" domain (header-only NVTX3: without an attached profiler every
// push and pop is a no-op after one environment check).  Names:
//   reference_build        sicp_set_reference: voxel grid, seed map
//   register               one registration run (sicp_register, _continue, sicp_resume)
//   sample                 minibatch draw (Sec. III-B)
//   transform_nn_gradient  transform, nearest neighbours, ICP gradient (Eqs. correspondences,
//                          trans_gradient / rotation_gradient)
//   telemetry              the run's per-iteration telemetry rows
//   stein_adam             bandwidths, Stein direction, Adam (Eq. stein_icp_phi, Sec. V)
//   moments                particle mean and covariance
//   graph_launch           launch of the captured run
//   nn, batched, surrogate_train: sicp_nn, sicp_register_batched, the learned field's training
// In a captured run the stage ranges enclose the capture, not the GPU work;
// with SICP_NO_GRAPH set they enclose each stage's launches.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace sicp {

inline nvtxDomainHandle_t nvtx_domain() {
    static nvtxDomainHandle_t d = nvtxDomainCreateA("steinicp");
    return d;
}

struct NvtxRange {
    explicit NvtxRange(const char* name) {
        nvtxEventAttributes_t a = {};
        a.version = NVTX_VERSION;
        a.size = NVTX_EVENT_ATTRIB_STRUCT_SIZE;
        a.messageType = NVTX_MESSAGE_TYPE_ASCII;
        a.message.ascii = name;
        nvtxDomainRangePushEx(nvtx_domain(), &a);
    }
    ~NvtxRange() { nvtxDomainRangePop(nvtx_domain()); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace sicp
