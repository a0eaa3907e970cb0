// lf2_io.cu -- binary snapshots of a field in LATfield2's write/read format (Sec. 3.5): one
// file, no header, the sites in row-major order (x fastest), each site's components next to
// each other.  Values are written in the field's storage precision (double or float), so a
// snapshot restores the state exactly; the Kahan compensation of an FP32+Kahan phi field can
// be written and read the same way for an exact restart.  Data go through a pinned staging
// buffer in chunks, so a field of any size needs only the chunk in host memory.
#include <cuda_runtime.h>

#include <cstdio>

#include "lf2_handles.h"

using namespace lf2;

namespace {

constexpr size_t kChunk = 64ull << 20;  // bytes per staging chunk

void *buffer_of(lf2_field f, int which) {
    switch (which) {
        case 0: return f->val[f->front];
        case 2: return f->comp[f->cfront];
        default: return nullptr;
    }
}

size_t elem_bytes(lf2_field f, int which) { return which == 2 ? sizeof(float) : f->esize; }

}  // namespace

extern "C" {

lf2_status lf2_field_write(lf2_field f, int which, const char *path, void *stream) {
    if (!f || !path) return set_error(LF2_ERR_INVALID, "NULL argument");
    if (which != 0 && which != 2) return set_error(LF2_ERR_INVALID, "which must be 0 (values) or 2 (compensation)");
    void *src = buffer_of(f, which);
    if (!src) return set_error(LF2_ERR_STATE, "the field has no compensation buffer");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t total = (size_t)f->count * elem_bytes(f, which);
    FILE *fp = fopen(path, "wb");
    if (!fp) return set_error(LF2_ERR_INVALID, "cannot open %s for writing", path);
    void *stage = nullptr;
    cudaError_t e = cudaMallocHost(&stage, total < kChunk ? (total ? total : 1) : kChunk);
    lf2_status st = LF2_OK;
    if (e != cudaSuccess) st = cuda_error(e, "cudaMallocHost(write staging)");
    for (size_t off = 0; st == LF2_OK && off < total; off += kChunk) {
        const size_t n = total - off < kChunk ? total - off : kChunk;
        e = cudaMemcpyAsync(stage, (const char *)src + off, n, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess)
            st = cuda_error(e, "snapshot copy");
        else if (fwrite(stage, 1, n, fp) != n)
            st = set_error(LF2_ERR_INVALID, "short write to %s", path);
    }
    if (stage) cudaFreeHost(stage);
    if (fclose(fp) != 0 && st == LF2_OK) st = set_error(LF2_ERR_INVALID, "closing %s failed", path);
    return st;
}

lf2_status lf2_field_read(lf2_field f, int which, const char *path, void *stream) {
    if (!f || !path) return set_error(LF2_ERR_INVALID, "NULL argument");
    if (which != 0 && which != 2) return set_error(LF2_ERR_INVALID, "which must be 0 (values) or 2 (compensation)");
    cudaStream_t s = (cudaStream_t)stream;
    if (which == 2) {
        if (f->prec != LF2_F32_KAHAN) return set_error(LF2_ERR_INVALID, "only LF2_F32_KAHAN fields have a compensation");
        lf2_status st = ensure_dynamic(f, s);  // allocates the compensation if missing
        if (st != LF2_OK) return st;
    }
    void *dst = buffer_of(f, which);
    const size_t total = (size_t)f->count * elem_bytes(f, which);
    FILE *fp = fopen(path, "rb");
    if (!fp) return set_error(LF2_ERR_INVALID, "cannot open %s", path);
    fseek(fp, 0, SEEK_END);
    const long size = ftell(fp);
    fseek(fp, 0, SEEK_SET);
    if (size < 0 || (size_t)size != total) {
        fclose(fp);
        return set_error(LF2_ERR_INVALID, "%s holds %ld bytes, the field needs %zu", path, size, total);
    }
    void *stage = nullptr;
    cudaError_t e = cudaMallocHost(&stage, total < kChunk ? (total ? total : 1) : kChunk);
    lf2_status st = LF2_OK;
    if (e != cudaSuccess) st = cuda_error(e, "cudaMallocHost(read staging)");
    for (size_t off = 0; st == LF2_OK && off < total; off += kChunk) {
        const size_t n = total - off < kChunk ? total - off : kChunk;
        if (fread(stage, 1, n, fp) != n) {
            st = set_error(LF2_ERR_INVALID, "short read from %s", path);
            break;
        }
        e = cudaMemcpyAsync((char *)dst + off, stage, n, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_error(e, "snapshot copy");
    }
    if (stage) cudaFreeHost(stage);
    fclose(fp);
    // a value snapshot without its compensation starts a fresh compensation
    if (st == LF2_OK && which == 0 && f->comp[f->cfront]) {
        e = cudaMemsetAsync(f->comp[f->cfront], 0, (size_t)f->count * sizeof(float), s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_error(e, "reset compensation");
    }
    return st;
}

}  // extern "C"
