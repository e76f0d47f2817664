// sf_multiframe.cuh -- launchers of the multiframe kernels (sf_multiframe.cu).
#pragma once
#include "sf_device.cuh"

// most elements of a frame that COALESCE sorts in one CTA
#define SF_MF_MAXK 8192

// one candidate pair: the element that becomes the new frame's element, the
// i-power d of a_r = i^d a_j, and the rows e on which the two phase vectors differ
struct MfPair {
    uint32_t owner, d;
    uint64_t e;
};

size_t sf_mf_pair_smem_bytes(uint64_t k);
cudaError_t sf_launch_mf_pair(const SfDev& d, int buf, int stage, uint64_t k, double tol, MfPair* pairs,
                              uint32_t* keep, uint32_t* counts, cudaStream_t s);
cudaError_t sf_launch_mf_gather(const SfDev& dst, int dst_buf, const uint64_t* ssig, const double2* samp,
                                const uint32_t* idx, uint32_t m, double scale, cudaStream_t s);
cudaError_t sf_launch_mf_import(const SfDev& dst, int dst_buf, uint64_t off, const uint64_t* xsig,
                                const double2* xamp, uint32_t m, cudaStream_t s);
