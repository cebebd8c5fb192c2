// segments.cu -- mfa_render_segments: the render with the paper's object-space
// decomposition (Sec. IV-A.1 partitioning, Sec. IV-A.4 per-block MFA-VV, Sec. IV-A.5
// compositing with the associative over) on one GPU.  The volume is split into a grid of
// equal blocks; one launch renders every block's ray segments into its own partial image
// (device staging from the library's pool), a second merges the partial images per pixel,
// nearest segment first.
#include "host.cuh"

using namespace mfa;

extern "C" int mfa_render_segments(const mfa_model* m, const mfa_camera* cam, const mfa_transfer_fn* tf, int width,
                                   int height, int n_samples, const int blocks[3], float* rgba_out,
                                   const mfa_render_opts* opts)
{
    if (!blocks) return fail(MFA_ERR_ARG, "blocks is NULL");
    for (int a = 0; a < 3; ++a)
        if (blocks[a] < 1 || blocks[a] > 64) return fail(MFA_ERR_ARG, "blocks[%d] = %d outside 1..64", a, blocks[a]);
    const int nb = blocks[0] * blocks[1] * blocks[2];
    if (nb > 64) return fail(MFA_ERR_ARG, "%d blocks: at most 64", nb);
    const int variant = opts ? opts->variant : 0;
    const int shape = opts ? opts->tile_shape : 0;
    if (variant != 0 && variant != 4 && variant != 6)
        return fail(MFA_ERR_ARG, "render variant %d: segments use 0, 4 or 6", variant);
    if (shape < 0 || shape >= kTileShapes) return fail(MFA_ERR_ARG, "tile_shape %d outside 0..%d", shape, kTileShapes - 1);
    RenderParams P;
    if (int rc = setup_render(m, cam, tf, width, height, n_samples, rgba_out, opts ? opts->samples_out : nullptr, P.s,
                              P.tf))
        return rc;
    cudaMemPool_t pool = nullptr;
    cudaError_t e = staging_pool(m->device, &pool);
    if (e != cudaSuccess) return cuda_fail(e, "staging pool");
    cudaStream_t st = current_stream();
    const size_t bytes = sizeof(float4) * static_cast<size_t>(nb) * width * height;
    float4* partial = nullptr;
    if ((e = cudaMallocFromPoolAsync(reinterpret_cast<void**>(&partial), bytes, pool, st)) != cudaSuccess)
        return cuda_fail(e, "partial images");
    e = launch_render_segments(m->dev, P, variant, shape, blocks, partial, st);
    if (e == cudaSuccess) e = launch_merge_segments(P.s, blocks, partial, st);
    cudaError_t ef = cudaFreeAsync(partial, st);
    if (e != cudaSuccess) return cuda_fail(e, "segment launch");
    if (ef != cudaSuccess) return cuda_fail(ef, "partial images free");
    return MFA_OK;
}
