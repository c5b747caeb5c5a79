// Save / load of a compressed matrix: the paper notes F can be assembled once
// and reused (Sections 1 and 9); this is the file format for that reuse.
//
// Layout (little-endian):
//   header  "VFHMAT01", u32 version, then a fixed record of sizes
//   sections perm, blocks, tile_first, tile_count, val, aux; each section is
//            u64 byte length, the bytes, u32 CRC-32 (IEEE 802.3 polynomial)
// Load rejects a wrong magic/version, a short file or a CRC mismatch.
#include <cstdio>
#include <cstring>
#include <memory>

#include "vf_hmat.cuh"

namespace vf {

static uint32_t crc_table[256];
static bool crc_init = false;

static void make_crc_table() {
    for (uint32_t i = 0; i < 256; ++i) {
        uint32_t c = i;
        for (int k = 0; k < 8; ++k) c = (c & 1u) ? 0xEDB88320u ^ (c >> 1) : c >> 1;
        crc_table[i] = c;
    }
    crc_init = true;
}

uint32_t crc32(const void* data, size_t n) {
    if (!crc_init) make_crc_table();
    const unsigned char* p = (const unsigned char*)data;
    uint32_t c = 0xFFFFFFFFu;
    for (size_t i = 0; i < n; ++i) c = crc_table[(c ^ p[i]) & 0xFFu] ^ (c >> 8);
    return c ^ 0xFFFFFFFFu;
}

struct FileHeader {
    char magic[8];
    uint32_t version;
    uint32_t tree_kind;
    int64_t nf;
    double tol;
    int64_t nblocks, n_val, n_aux, n_T, ntiles;
    int32_t max_q;
    uint32_t flags;  // bit0 bf16, bit1 fp8
    int64_t n_hier;
    vf_assemble_stats stats;
};

static const uint32_t kVersion = 2;  // 2: assembly statistics with the predictor audits

static bool write_section(FILE* f, const void* p, uint64_t bytes) {
    uint32_t c = crc32(p, bytes);
    return fwrite(&bytes, 8, 1, f) == 1 && (bytes == 0 || fwrite(p, 1, bytes, f) == bytes) && fwrite(&c, 4, 1, f) == 1;
}

static vf_status read_section(FILE* f, void* p, uint64_t expect) {
    uint64_t bytes;
    uint32_t c;
    VF_CHECK(fread(&bytes, 8, 1, f) == 1, VF_E_CORRUPT, "vf_hmat_load: truncated section header");
    VF_CHECK(bytes == expect, VF_E_CORRUPT, "vf_hmat_load: section has %llu bytes, expected %llu",
             (unsigned long long)bytes, (unsigned long long)expect);
    VF_CHECK(bytes == 0 || fread(p, 1, bytes, f) == bytes, VF_E_CORRUPT, "vf_hmat_load: truncated section");
    VF_CHECK(fread(&c, 4, 1, f) == 1, VF_E_CORRUPT, "vf_hmat_load: truncated CRC");
    VF_CHECK(c == crc32(p, bytes), VF_E_CORRUPT, "vf_hmat_load: CRC mismatch");
    return VF_OK;
}

__global__ void k_to_bf16_io(const float* __restrict__ x, __nv_bfloat16* __restrict__ y, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16_rn(x[i]);
}

__global__ void k_to_fp8_io(const HBlock* __restrict__ blocks, const float* __restrict__ x,
                            __nv_fp8_e4m3* __restrict__ y, const float* __restrict__ scales) {
    const HBlock b = blocks[blockIdx.x];
    int64_t len = 0;
    if (b.kind == VF_BLK_DENSE) len = (int64_t)b.m * b.n;
    else if (b.kind == VF_BLK_CSR) len = b.m1;
    else if (b.kind == VF_BLK_SVD) len = (int64_t)(b.m1 + b.n1) * b.q;
    float inv = 1.f / scales[blockIdx.x];
    for (int64_t i = threadIdx.x; i < len; i += blockDim.x) y[b.off_val + i] = __nv_fp8_e4m3(x[b.off_val + i] * inv);
}

}  // namespace vf

using namespace vf;

extern "C" vf_status vf_hmat_save(const vf_hmat* h, const char* path) {
    clear_error();
    VF_CHECK(h && path, VF_E_INVAL, "vf_hmat_save: null argument");
    device_guard g(h->device);
    std::vector<float> val;
    std::vector<int32_t> aux;
    VF_TRY(h->val.download(val));
    VF_TRY(h->aux.download(aux));
    val.resize(h->n_val);
    aux.resize(h->n_aux);
    std::vector<float> sc8;
    if (h->has_fp8) VF_TRY(h->scale8.download(sc8));
    FILE* f = fopen(path, "wb");
    VF_CHECK(f, VF_E_IO, "vf_hmat_save: cannot open %s", path);
    FileHeader hd{};
    memcpy(hd.magic, "VFHMAT01", 8);
    hd.version = kVersion;
    hd.tree_kind = (uint32_t)h->tree_kind;
    hd.nf = h->nf;
    hd.tol = h->tol;
    hd.nblocks = (int64_t)h->h_blocks.size();
    hd.n_val = h->n_val;
    hd.n_aux = h->n_aux;
    hd.n_T = h->n_T;
    hd.ntiles = (int64_t)h->h_tile_first.size();
    hd.max_q = h->max_q;
    hd.flags = (h->has_bf16 ? 1u : 0u) | (h->has_fp8 ? 2u : 0u);
    hd.n_hier = h->n_hier;
    hd.stats = h->stats;
    bool ok = fwrite(&hd, sizeof(hd), 1, f) == 1;
    ok = ok && write_section(f, h->h_perm.data(), h->h_perm.size() * 4);
    ok = ok && write_section(f, h->h_blocks.data(), h->h_blocks.size() * sizeof(HBlock));
    ok = ok && write_section(f, h->h_tile_first.data(), h->h_tile_first.size() * 4);
    ok = ok && write_section(f, h->h_tile_count.data(), h->h_tile_count.size() * 4);
    ok = ok && write_section(f, val.data(), val.size() * 4);
    ok = ok && write_section(f, aux.data(), aux.size() * 4);
    ok = ok && write_section(f, sc8.data(), h->has_fp8 ? h->h_blocks.size() * 4 : 0);
    ok = (fclose(f) == 0) && ok;
    VF_CHECK(ok, VF_E_IO, "vf_hmat_save: write to %s failed", path);
    return VF_OK;
}

extern "C" vf_status vf_hmat_load(const char* path, int32_t device, vf_hmat** out) {
    clear_error();
    VF_CHECK(path && out, VF_E_INVAL, "vf_hmat_load: null argument");
    *out = nullptr;
    FILE* f = fopen(path, "rb");
    VF_CHECK(f, VF_E_IO, "vf_hmat_load: cannot open %s", path);
    std::unique_ptr<FILE, int (*)(FILE*)> guard(f, fclose);
    FileHeader hd{};
    VF_CHECK(fread(&hd, sizeof(hd), 1, f) == 1, VF_E_CORRUPT, "vf_hmat_load: truncated header");
    VF_CHECK(memcmp(hd.magic, "VFHMAT01", 8) == 0, VF_E_CORRUPT, "vf_hmat_load: bad magic");
    VF_CHECK(hd.version == kVersion, VF_E_CORRUPT, "vf_hmat_load: unsupported version %u", hd.version);
    VF_CHECK(hd.nf > 0 && hd.nblocks >= 0 && hd.n_val >= 0 && hd.n_aux >= 0 && hd.ntiles > 0 && hd.nf < (1ll << 31),
             VF_E_CORRUPT, "vf_hmat_load: implausible sizes");
    device_guard g(device);
    VF_TRY_CUDA(cudaSetDevice(device));
    auto H = std::make_unique<vf_hmat>();
    H->device = device;
    H->nf = hd.nf;
    H->tol = hd.tol;
    H->tree_kind = (int)hd.tree_kind;
    H->n_val = hd.n_val;
    H->n_aux = hd.n_aux;
    H->n_T = hd.n_T;
    H->max_q = hd.max_q;
    H->n_hier = hd.n_hier;
    H->stats = hd.stats;
    H->h_perm.resize(hd.nf);
    H->h_blocks.resize(hd.nblocks);
    H->h_tile_first.resize(hd.ntiles);
    H->h_tile_count.resize(hd.ntiles);
    std::vector<float> val(hd.n_val);
    std::vector<int32_t> aux(hd.n_aux);
    std::vector<float> sc8((hd.flags & 2u) ? hd.nblocks : 0);
    VF_TRY(read_section(f, H->h_perm.data(), hd.nf * 4));
    VF_TRY(read_section(f, H->h_blocks.data(), hd.nblocks * sizeof(HBlock)));
    VF_TRY(read_section(f, H->h_tile_first.data(), hd.ntiles * 4));
    VF_TRY(read_section(f, H->h_tile_count.data(), hd.ntiles * 4));
    VF_TRY(read_section(f, val.data(), hd.n_val * 4));
    VF_TRY(read_section(f, aux.data(), hd.n_aux * 4));
    VF_TRY(read_section(f, sc8.data(), sc8.size() * 4));
    // structural checks before anything reaches the device
    std::vector<char> seen(hd.nf, 0);
    for (int32_t p : H->h_perm) {
        VF_CHECK(p >= 0 && p < hd.nf && !seen[p], VF_E_CORRUPT, "vf_hmat_load: permutation is not a bijection");
        seen[p] = 1;
    }
    for (const HBlock& b : H->h_blocks) {
        VF_CHECK(b.r0 >= 0 && b.m > 0 && b.r0 + (int64_t)b.m <= hd.nf && b.c0 >= 0 && b.n > 0 &&
                     b.c0 + (int64_t)b.n <= hd.nf && b.off_val >= 0 && b.off_val <= hd.n_val && b.off_aux >= 0 &&
                     b.off_aux <= hd.n_aux,
                 VF_E_CORRUPT, "vf_hmat_load: block out of range");
        VF_CHECK(b.kind == VF_BLK_DENSE || b.kind == VF_BLK_CSR || b.kind == VF_BLK_SVD, VF_E_CORRUPT,
                 "vf_hmat_load: bad block kind");
    }
    VF_TRY(H->perm.upload(H->h_perm));
    std::vector<int32_t> ip(hd.nf);
    for (int64_t k = 0; k < hd.nf; ++k) ip[H->h_perm[k]] = (int32_t)k;
    VF_TRY(H->iperm.upload(ip));
    VF_TRY(H->blocks.upload(H->h_blocks));
    // pools are padded by 16 elements: the multiply copies 16-byte aligned supersets
    val.resize(hd.n_val + 16, 0.f);
    VF_TRY(H->val.upload(val));
    aux.resize(hd.n_aux + 16, 0);
    VF_TRY(H->aux.upload(aux));
    if (hd.flags & 1u) {
        VF_TRY(H->val16.alloc(val.size()));
        k_to_bf16_io<<<1024, 256>>>(H->val.p, H->val16.p, (int64_t)val.size());
        VF_TRY_CUDA(cudaGetLastError());
        H->has_bf16 = true;
    }
    if ((hd.flags & 2u) && hd.nblocks > 0) {
        VF_TRY(H->val8.alloc(val.size()));
        VF_TRY(H->scale8.upload(sc8));
        VF_TRY_CUDA(cudaMemset(H->val8.p, 0, val.size()));
        k_to_fp8_io<<<(unsigned)hd.nblocks, 256>>>(H->blocks.p, H->val.p, H->val8.p, H->scale8.p);
        VF_TRY_CUDA(cudaGetLastError());
        H->has_fp8 = true;
    }
    VF_TRY_CUDA(cudaDeviceSynchronize());
    VF_TRY(H->upload_all());
    *out = H.release();
    return VF_OK;
}

// The block-diagonal composition diag(F_1, ..., F_k) of several matrices:
// stacked facet (and tree) numbering mesh after mesh, every block shifted
// to its mesh's rows and columns, the payload pools concatenated (column
// and row indices in the pools shifted the same way), one segment per
// mesh.  Multiplies and solves of the result run every mesh in the same
// launches, over one work list of all meshes' row tiles.
extern "C" vf_status vf_hmat_stack(const vf_hmat* const* F, int32_t nmeshes, vf_hmat** out) {
    clear_error();
    VF_CHECK(F && out && nmeshes >= 1, VF_E_INVAL, "vf_hmat_stack: null argument");
    *out = nullptr;
    for (int32_t k = 0; k < nmeshes; ++k) {
        VF_CHECK(F[k], VF_E_INVAL, "vf_hmat_stack: null matrix %d", (int)k);
        VF_CHECK(F[k]->device == F[0]->device, VF_E_INVAL, "vf_hmat_stack: matrices on different devices");
    }
    device_guard g(F[0]->device);
    auto H = std::make_unique<vf_hmat>();
    H->device = F[0]->device;
    H->tree_kind = F[0]->tree_kind;
    H->has_bf16 = H->has_fp8 = true;
    int64_t nf = 0, nv = 0, na = 0, nT = 0;
    std::vector<int32_t> aux_all;
    std::vector<float> sc8;
    H->h_seg_row0.push_back(0);
    H->h_seg_tile0.push_back(0);
    for (int32_t k = 0; k < nmeshes; ++k) {
        const vf_hmat* f = F[k];
        VF_CHECK(nf + f->nf < (1ll << 31), VF_E_INVAL, "vf_hmat_stack: more than 2^31 facets");
        H->tol = std::max(H->tol, f->tol);
        H->has_bf16 = H->has_bf16 && f->has_bf16;
        H->has_fp8 = H->has_fp8 && f->has_fp8;
        std::vector<int32_t> a;
        if (f->n_aux > 0) VF_TRY(f->aux.download(a));
        a.resize(f->n_aux);
        for (const HBlock& b : f->h_blocks) {
            HBlock c = b;
            c.r0 += (int32_t)nf;
            c.c0 += (int32_t)nf;
            c.off_val += nv;
            c.off_aux += na;
            if (c.off_T >= 0) c.off_T += nT;
            H->h_blocks.push_back(c);
            // tree-order indices stored in the pool: CSR columns, SVD rows and columns
            if (b.kind == VF_BLK_CSR)
                for (int64_t z = b.off_aux + b.m + 1; z < b.off_aux + b.m + 1 + b.m1; ++z) a[z] += (int32_t)nf;
            else if (b.kind == VF_BLK_SVD)
                for (int64_t z = b.off_aux; z < b.off_aux + b.m1 + b.n1; ++z) a[z] += (int32_t)nf;
        }
        aux_all.insert(aux_all.end(), a.begin(), a.end());
        for (int32_t p : f->h_perm) H->h_perm.push_back(p + (int32_t)nf);
        for (size_t t = 0; t < f->h_tile_first.size(); ++t) {
            H->h_tile_first.push_back(f->h_tile_first[t] + (int32_t)nf);
            H->h_tile_count.push_back(f->h_tile_count[t]);
        }
        if (f->has_fp8) {
            std::vector<float> s;
            VF_TRY(f->scale8.download(s));
            s.resize(f->h_blocks.size());
            sc8.insert(sc8.end(), s.begin(), s.end());
        }
        H->max_q = std::max(H->max_q, f->max_q);
        H->n_hier += f->n_hier;
        vf_assemble_stats& S = H->stats;
        for (int i = 0; i < 5; ++i) S.nblocks[i] += f->stats.nblocks[i], S.bytes[i] += f->stats.bytes[i];
        S.nnz_visible += f->stats.nnz_visible;
        S.probes += f->stats.probes;
        S.probes_failed += f->stats.probes_failed;
        S.probes_skipped += f->stats.probes_skipped;
        S.probes_predicted_skip += f->stats.probes_predicted_skip;
        S.predictor_audits += f->stats.predictor_audits;
        S.predictor_audit_wins += f->stats.predictor_audit_wins;
        S.predictor_fallbacks += f->stats.predictor_fallbacks;
        S.verify_failed += f->stats.verify_failed;
        S.max_rank = std::max(S.max_rank, f->stats.max_rank);
        nf += f->nf;
        nv += f->n_val;
        na += f->n_aux;
        nT += f->n_T;
        H->h_seg_row0.push_back((int32_t)nf);
        H->h_seg_tile0.push_back((int32_t)H->h_tile_first.size());
    }
    H->nf = nf;
    H->n_val = nv;
    H->n_aux = na;
    H->n_T = nT;
    // pools are padded by 16 elements: the multiply copies 16-byte aligned supersets
    VF_TRY(H->val.alloc(nv + 16));
    VF_TRY_CUDA(cudaMemset(H->val.p, 0, (nv + 16) * sizeof(float)));
    if (H->has_bf16) {
        VF_TRY(H->val16.alloc(nv + 16));
        VF_TRY_CUDA(cudaMemset(H->val16.p, 0, (nv + 16) * sizeof(__nv_bfloat16)));
    }
    if (H->has_fp8) {
        VF_TRY(H->val8.alloc(nv + 16));
        VF_TRY_CUDA(cudaMemset(H->val8.p, 0, nv + 16));
        VF_TRY(H->scale8.upload(sc8));
    }
    for (int64_t k = 0, o = 0; k < nmeshes; o += F[k]->n_val, ++k) {
        const vf_hmat* f = F[k];
        if (f->n_val == 0) continue;
        VF_TRY_CUDA(cudaMemcpy(H->val.p + o, f->val.p, f->n_val * sizeof(float), cudaMemcpyDeviceToDevice));
        if (H->has_bf16)
            VF_TRY_CUDA(cudaMemcpy(H->val16.p + o, f->val16.p, f->n_val * sizeof(__nv_bfloat16),
                                   cudaMemcpyDeviceToDevice));
        if (H->has_fp8) VF_TRY_CUDA(cudaMemcpy(H->val8.p + o, f->val8.p, f->n_val, cudaMemcpyDeviceToDevice));
    }
    aux_all.resize(na + 16, 0);
    VF_TRY(H->aux.upload(aux_all));
    VF_TRY(H->perm.upload(H->h_perm));
    std::vector<int32_t> ip(nf);
    for (int64_t k = 0; k < nf; ++k) ip[H->h_perm[k]] = (int32_t)k;
    VF_TRY(H->iperm.upload(ip));
    VF_TRY(H->blocks.upload(H->h_blocks));
    VF_TRY(H->upload_all());
    *out = H.release();
    return VF_OK;
}

extern "C" int32_t vf_hmat_nsegments(const vf_hmat* h) { return h ? h->nseg() : -1; }
