// Block-structured particle files (Section 3.1): a file is an n x N array of
// floats, one contiguous block of N values per particle property.  A reader
// takes the same slice of every block it needs (the n x N/nprocs subarray of
// one process) and converts the byte order when the file's differs from the
// host's.  The loader streams slices to device arrays from host threads of
// its own, each through two pinned staging buffers, so reading overlaps the
// copies and the device work of other streams.  Host code only.
#include <fcntl.h>
#include <unistd.h>

#include <cerrno>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "splotch.h"

namespace {

bool host_big_endian() {
    const uint32_t one = 1;
    unsigned char first;
    std::memcpy(&first, &one, 1);
    return first == 0;
}

void swap_bytes(float *p, size_t n) {
    for (size_t i = 0; i < n; ++i) {
        uint32_t w;
        std::memcpy(&w, p + i, 4);
        w = __builtin_bswap32(w);
        std::memcpy(p + i, &w, 4);
    }
}

// The slice [first, first + count) of block `block` lies inside the file description.
bool slice_ok(const splotch_block_file *f, int32_t block, uint64_t first, uint64_t count) {
    if (!f || !f->path || f->n_blocks < 1 || block < 0 || block >= f->n_blocks) return false;
    if (first > f->n_particles || count > f->n_particles - first) return false;
    if (f->n_particles > (UINT64_MAX - f->offset) / 4 / (uint64_t)f->n_blocks) return false;
    return true;
}

// pread the slice (restarting after partial reads and interrupts), then fix the byte order.
int read_slice(int fd, const splotch_block_file *f, int32_t block, uint64_t first, uint64_t count, float *dst) {
    const uint64_t at = f->offset + 4 * ((uint64_t)block * f->n_particles + first);
    char *out = reinterpret_cast<char *>(dst);
    uint64_t done = 0, want = 4 * count;
    while (done < want) {
        const ssize_t r = pread(fd, out + done, (size_t)(want - done), (off_t)(at + done));
        if (r < 0 && errno == EINTR) continue;
        if (r <= 0) return SPLOTCH_ERR_IO;   // error, or the file ends before the slice
        done += (uint64_t)r;
    }
    if ((f->big_endian != 0) != host_big_endian()) swap_bytes(dst, count);
    return SPLOTCH_OK;
}

}  // namespace

// One reader thread's staging: two pinned buffers and the events that mark
// the end of the copies reading them.
struct Stage {
    float *buf[2] = {nullptr, nullptr};
    cudaEvent_t ev[2] = {nullptr, nullptr};
};

struct splotch_loader {
    int device = 0;
    size_t chunk = 0;
    std::vector<Stage> stage;        // one per reader thread
    std::vector<std::thread> workers;
    std::vector<int> wstatus;
    bool running = false;
    // the current load, copied at start
    splotch_block_file file{};
    std::string path;
    std::vector<int32_t> blocks;
    std::vector<float *> dst;
    uint64_t first = 0, count = 0;
    cudaStream_t stream = nullptr;

    // Reader t takes chunks t, t + T, t + 2T, ... of the load (chunks run
    // block by block), alternating between its two buffers.
    void run(int t) {
        int &status = wstatus[t];
        if (cudaSetDevice(device) != cudaSuccess) {
            status = SPLOTCH_ERR_CUDA;
            return;
        }
        const int fd = open(path.c_str(), O_RDONLY);
        if (fd < 0) {
            status = SPLOTCH_ERR_IO;
            return;
        }
        const uint64_t per = chunk / 4;
        const uint64_t per_block = (count + per - 1) / per;
        const uint64_t total = per_block * dst.size();
        const uint64_t T = stage.size();
        Stage &S = stage[t];
        int b = 0;
        for (uint64_t c = (uint64_t)t; c < total; c += T) {
            const size_t d = (size_t)(c / per_block);
            const uint64_t off = (c % per_block) * per;
            const uint64_t m = count - off < per ? count - off : per;
            // the copy that last used this buffer has to be done before it is refilled
            if (cudaEventSynchronize(S.ev[b]) != cudaSuccess) {
                status = SPLOTCH_ERR_CUDA;
                break;
            }
            const int st = read_slice(fd, &file, blocks[d], first + off, m, S.buf[b]);
            if (st != SPLOTCH_OK) {
                status = st;
                break;
            }
            if (cudaMemcpyAsync(dst[d] + off, S.buf[b], 4 * m, cudaMemcpyHostToDevice, stream) != cudaSuccess ||
                cudaEventRecord(S.ev[b], stream) != cudaSuccess) {
                status = SPLOTCH_ERR_CUDA;
                break;
            }
            b ^= 1;
        }
        close(fd);
    }
};

extern "C" {

int splotch_block_read(const splotch_block_file *file, int32_t block, uint64_t first, uint64_t count, float *dst) {
    if (!slice_ok(file, block, first, count) || (count && !dst)) return SPLOTCH_ERR_ARG;
    if (count == 0) return SPLOTCH_OK;
    const int fd = open(file->path, O_RDONLY);
    if (fd < 0) return SPLOTCH_ERR_IO;
    const int st = read_slice(fd, file, block, first, count, dst);
    close(fd);
    return st;
}

int splotch_loader_create(size_t chunk_bytes, int32_t n_threads, splotch_loader **out) {
    if (!out || chunk_bytes < 4096 || chunk_bytes % 4 || n_threads < 1 || n_threads > 64) return SPLOTCH_ERR_ARG;
    *out = nullptr;
    splotch_loader *L = new splotch_loader();
    L->chunk = chunk_bytes;
    L->stage.resize((size_t)n_threads);
    bool ok = cudaGetDevice(&L->device) == cudaSuccess;
    for (Stage &S : L->stage)
        for (int b = 0; b < 2 && ok; ++b) {
            ok = cudaHostAlloc(reinterpret_cast<void **>(&S.buf[b]), chunk_bytes, cudaHostAllocDefault) == cudaSuccess;
            ok = ok && cudaEventCreateWithFlags(&S.ev[b], cudaEventDisableTiming) == cudaSuccess;
        }
    if (!ok) {
        for (Stage &S : L->stage)
            for (int b = 0; b < 2; ++b) {
                if (S.buf[b]) cudaFreeHost(S.buf[b]);
                if (S.ev[b]) cudaEventDestroy(S.ev[b]);
            }
        delete L;
        return SPLOTCH_ERR_CUDA;
    }
    *out = L;
    return SPLOTCH_OK;
}

int splotch_loader_start(splotch_loader *L, const splotch_block_file *file, int32_t n_dst, const int32_t *blocks,
                         uint64_t first, uint64_t count, float *const *dst, void *stream) {
    if (!L || L->running || n_dst < 0 || (n_dst && (!blocks || !dst))) return SPLOTCH_ERR_ARG;
    for (int32_t d = 0; d < n_dst; ++d)
        if (!slice_ok(file, blocks[d], first, count) || (count && !dst[d])) return SPLOTCH_ERR_ARG;
    if (n_dst == 0 && !slice_ok(file, 0, first, count)) return SPLOTCH_ERR_ARG;
    L->file = *file;
    L->path = file->path;
    L->file.path = L->path.c_str();
    L->blocks.assign(blocks, blocks + n_dst);
    L->dst.assign(dst, dst + n_dst);
    L->first = first;
    L->count = count;
    L->stream = static_cast<cudaStream_t>(stream);
    L->wstatus.assign(L->stage.size(), SPLOTCH_OK);
    L->running = true;
    L->workers.clear();
    for (size_t t = 0; t < L->stage.size(); ++t) L->workers.emplace_back([L, t] { L->run((int)t); });
    return SPLOTCH_OK;
}

int splotch_loader_wait(splotch_loader *L) {
    if (!L) return SPLOTCH_ERR_ARG;
    if (L->running) {
        for (std::thread &w : L->workers) w.join();
        L->workers.clear();
        L->running = false;
    }
    for (int st : L->wstatus)
        if (st != SPLOTCH_OK) return st;
    return SPLOTCH_OK;
}

int splotch_loader_destroy(splotch_loader *L) {
    if (!L) return SPLOTCH_ERR_ARG;
    splotch_loader_wait(L);
    int st = SPLOTCH_OK;
    for (Stage &S : L->stage)
        for (int b = 0; b < 2; ++b) {
            // copies still reading a staging buffer must finish before it is freed
            if (cudaEventSynchronize(S.ev[b]) != cudaSuccess) st = SPLOTCH_ERR_CUDA;
            cudaEventDestroy(S.ev[b]);
            cudaFreeHost(S.buf[b]);
        }
    delete L;
    return st;
}

}  // extern "C"
