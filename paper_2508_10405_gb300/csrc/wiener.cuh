// The Fourier form of the App. E deblurring filter (deblur.cu): per comb
// node a 2s x 2s block filtered by the Wiener ratio
// conj(F m'') F m_rtm / (|F m''|^2 + eps mean|F m''|^2), block results
// blk [2][nkz * nkx][4 s^2], blended with the bilinear valence. s <= 32.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

namespace lsrtm {

int wiener_max_spacing();
size_t wiener_smem(int s);
cudaError_t launch_wiener(const float *mref, const float *mrem, int nz, int nx, int s, double eps, float *blk,
                          float *out, cudaStream_t st);

}  // namespace lsrtm
