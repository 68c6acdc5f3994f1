// The interpolated PSF Hessian of App. D on 3D images (psfhess.cu): node
// windows of (2 half + 1)^3 voxels packed per (node, offset) as float4 over
// the four parameter blocks (component 2 i + j: output plane i, input plane
// j), and the application of P H P or P H^T P to a [2][nz][ny][nx] image with
// the eight-corner weights of Eq. (trilinear).
#pragma once

#include <cuda_runtime.h>

namespace lsrtm {

struct PsfHess3Dev {
    int nz, ny, nx, s, half, nkz, nky, nkx, mask;
    const float4 *pt;   // [nkz][nky][nkx][(2 half + 1)^3]
};

cudaError_t launch_psfh3_patches(const float *psf_vp, const float *psf_ip, const PsfHess3Dev &a, float4 *pt,
                                 cudaStream_t st);
cudaError_t launch_psfh3_apply(const PsfHess3Dev &a, bool transpose, const float *in, float *out, cudaStream_t s);

}  // namespace lsrtm
