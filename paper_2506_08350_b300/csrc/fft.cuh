// Raw launchers of the ASM / FFT kernels defined in fft.cu, taking explicit
// plans and tables (no context), for other translation units.
#pragma once
#include "common.cuh"

namespace hcgs {

struct HArgs {
    double lam[MAX_C];
    double z[MAX_L];
};

void factor_radices(int n, int* radix, int* nst);
// Column transforms of nplanes H x W planes (in place allowed); tw = twiddles of length H.
cudaError_t launch_fft_cols_raw(bool inverse, const float2* in, float2* out, int nplanes, int H, int W,
                                const FftPlanArg& plan, const float2* tw, float scale, cudaStream_t st);
// out[b][l][c] = IDFT_rows(conj(H) DFT_rows(in[b][c])); tw = twiddles of length W.
cudaError_t launch_rows_spread_conj_raw(const float2* in, float2* out, int B, int L, int C, int H, int W,
                                        const float2* hq, const FftPlanArg& plan, const float2* tw,
                                        cudaStream_t st);
cudaError_t launch_build_hq_raw(float2* hq, int H, int W, int C, int L, double px, double py, const HArgs& a,
                                int band_limit, cudaStream_t st);

}  // namespace hcgs
