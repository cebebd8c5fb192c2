// checkpoint.cu -- reading a model's control points back and writing / reading models to
// files (the paper stores each block's MFA model after encoding and reads it back for
// rendering, Sec. IV-A.2).  A file holds what defines the model exactly: the degrees,
// counts, storage type, FP64 knots and the stored control points; loading it creates a
// model whose stored values are bit-identical (rounding a value already in the storage
// type to that type is the identity).
//
// File layout (little-endian): a 64-byte header {char magic[8] = "MFAMODL1"; int32 version
// = 1; int32 degree[3]; int32 nctrl[3]; int32 storage; int32 reserved[6] = 0}, then the
// three knot vectors (n_d + p_d + 1 FP64 values each, x, y, z), then the control points
// [n_z][n_y][n_x] in the storage type (4 bytes FP32, 2 bytes FP16 / BF16).
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>

#include "host.cuh"

namespace mfa {
namespace {

struct FileHeader {
    char magic[8];
    int32_t version;
    int32_t degree[3];
    int32_t nctrl[3];
    int32_t storage;
    int32_t reserved[6];
};
static_assert(sizeof(FileHeader) == 64, "the file header is 64 bytes");
constexpr char kMagic[8] = { 'M', 'F', 'A', 'M', 'O', 'D', 'L', '1' };

size_t storage_bytes(int storage) { return storage == MFA_F32 ? 4 : 2; }

}  // namespace
}  // namespace mfa

using namespace mfa;

extern "C" int mfa_model_get_ctrl(const mfa_model* m, void* host_out)
{
    if (!m || !host_out) return fail(MFA_ERR_ARG, "model and host_out must be non-NULL");
    if (int rc = check_model_device(m)) return rc;
    const int nx = m->nctrl[0], ny = m->nctrl[1], nz = m->nctrl[2];
    const size_t bytes = static_cast<size_t>(nx) * ny * nz * storage_bytes(m->storage);
    // the plain array of stored values is the model's own copy: one device-to-host copy.
    // Compact models hold them only in their entries (the first S values of entry e are the
    // padded row's positions S e .. S e + S - 1, S the entry stride): a pitched copy of those
    // gives the padded plain array, trimmed here on the host.
    cudaStream_t st = current_stream();
    cudaError_t e;
    if (m->dev.raw) {
        e = cudaMemcpyAsync(host_out, m->dev.raw, bytes, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    } else {
        const size_t elem = storage_bytes(m->storage);
        const size_t nxp = m->dev.nxp, nyp = m->dev.nyp, nzp = m->dev.nzp;
        const size_t S = compact_stride(m->dev.q, m->dev.storage), V = compact_values(m->dev.storage);
        std::vector<unsigned char> padded(nxp * nyp * nzp * elem);
        e = cudaMemcpy2DAsync(padded.data(), S * elem, m->dev.win, V * elem, S * elem, nxp / S * nyp * nzp,
                              cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e == cudaSuccess) {
            unsigned char* dst = static_cast<unsigned char*>(host_out);
            for (size_t k = 0; k < static_cast<size_t>(nz); ++k)
                for (size_t j = 0; j < static_cast<size_t>(ny); ++j)
                    std::memcpy(dst + ((k * ny + j) * nx) * elem, padded.data() + ((k * nyp + j) * nxp) * elem, nx * elem);
        }
    }
    return e == cudaSuccess ? MFA_OK : cuda_fail(e, "read control points");
}

extern "C" int mfa_model_save(const mfa_model* m, const char* path)
{
    if (!m || !path) return fail(MFA_ERR_ARG, "model and path must be non-NULL");
    const size_t n = static_cast<size_t>(m->nctrl[0]) * m->nctrl[1] * m->nctrl[2];
    std::vector<unsigned char> ctrl(n * storage_bytes(m->storage));
    if (int rc = mfa_model_get_ctrl(m, ctrl.data())) return rc;
    FileHeader h;
    std::memset(&h, 0, sizeof h);
    std::memcpy(h.magic, kMagic, sizeof kMagic);
    h.version = 1;
    for (int a = 0; a < 3; ++a) {
        h.degree[a] = m->degree[a];
        h.nctrl[a] = m->nctrl[a];
    }
    h.storage = m->storage;
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(MFA_ERR_ARG, "cannot open %s for writing", path);
    bool ok = std::fwrite(&h, sizeof h, 1, f) == 1;
    for (int a = 0; a < 3 && ok; ++a)
        ok = std::fwrite(m->knots[a].data(), sizeof(double), m->knots[a].size(), f) == m->knots[a].size();
    ok = ok && std::fwrite(ctrl.data(), 1, ctrl.size(), f) == ctrl.size();
    ok = (std::fclose(f) == 0) && ok;
    return ok ? MFA_OK : fail(MFA_ERR_ARG, "cannot write %s", path);
}

extern "C" mfa_model* mfa_model_load(const char* path)
{
    if (!path) return fail(MFA_ERR_ARG, "path must be non-NULL"), nullptr;
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(MFA_ERR_ARG, "cannot open %s", path), nullptr;
    auto bad = [&](const char* why) -> mfa_model* {
        std::fclose(f);
        fail(MFA_ERR_ARG, "%s: %s", path, why);
        return nullptr;
    };
    FileHeader h;
    if (std::fread(&h, sizeof h, 1, f) != 1) return bad("shorter than the header");
    if (std::memcmp(h.magic, kMagic, sizeof kMagic) != 0) return bad("not an MFA model file");
    if (h.version != 1) return bad("unsupported version");
    if (h.storage != MFA_F32 && h.storage != MFA_F16 && h.storage != MFA_BF16) return bad("bad storage type");
    for (int a = 0; a < 3; ++a)
        if (h.degree[a] < 1 || h.degree[a] > kMaxDegree || h.nctrl[a] < h.degree[a] + 1 || h.nctrl[a] > (1 << 24))
            return bad("bad degree or control-point count");
    if (static_cast<long long>(h.nctrl[0] + kPad) * (h.nctrl[1] + kPad) * (h.nctrl[2] + kPad) >= (1LL << 31))
        return bad("model too large");
    std::vector<double> U[3];
    for (int a = 0; a < 3; ++a) {
        U[a].resize(static_cast<size_t>(h.nctrl[a]) + h.degree[a] + 1);
        if (std::fread(U[a].data(), sizeof(double), U[a].size(), f) != U[a].size()) return bad("truncated knots");
    }
    const size_t n = static_cast<size_t>(h.nctrl[0]) * h.nctrl[1] * h.nctrl[2];
    std::vector<unsigned char> ctrl(n * storage_bytes(h.storage));
    if (std::fread(ctrl.data(), 1, ctrl.size(), f) != ctrl.size()) return bad("truncated control points");
    unsigned char extra;
    if (std::fread(&extra, 1, 1, f) != 0) return bad("trailing bytes");
    std::fclose(f);
    const int degree[3] = { h.degree[0], h.degree[1], h.degree[2] };
    const int nctrl[3] = { h.nctrl[0], h.nctrl[1], h.nctrl[2] };
    const double* const knots[3] = { U[0].data(), U[1].data(), U[2].data() };
    const mfa_dtype st = static_cast<mfa_dtype>(h.storage);
    return model_create(degree, nctrl, knots, ctrl.data(), st, st, false);
}
