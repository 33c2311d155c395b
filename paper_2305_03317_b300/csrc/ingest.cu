// Graph ingest on the device: validation, degree-descending relabelling and
// the relabelled CSR with sorted rows.
//
// The paper's backend copies the CSR to the GPU once and keeps it there
// (Section 3.1; Section 4.3 on keeping transfers few).  Here the copy is also
// relabelled: new id r is the r-th vertex in (degree descending, original id
// ascending) order, so heavy rows form a prefix [0, n_heavy) and isolated
// vertices a suffix [n_nz, n).  Both sorts are one stable LSD radix sort of
// 64-bit keys over chosen 8-bit digit windows:
//   permutation: key = (0xFFFFFFFF - degree) << 32 | id, digits of the degree
//                part only (input is in id order and the sort is stable);
//   arcs:        key = new_row << 32 | new_col, column digits then row digits.
// Duplicates and self-loops show up in the sorted arc keys; symmetry is a
// binary search of every arc's reverse.
#include <cstdint>
#include <cuda_runtime.h>

#include "bc_internal.cuh"

namespace bcx {

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortIPT = 16;
constexpr int kTile = kSortThreads * kSortIPT;  // 4096 keys per block
constexpr int kSortWarps = kSortThreads / 32;

enum : int { V_OFFSETS = 1, V_RANGE = 2, V_SELF = 4, V_DUP = 8, V_ASYM = 16 };

__global__ void k_check_offsets(const int* off, int n, long long m, int* err) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0 && (off[0] != 0 || (long long)off[n] != m)) atomicOr(err, V_OFFSETS);
    if (i < n && off[i + 1] < off[i]) atomicOr(err, V_OFFSETS);
}

__global__ void k_check_range(const int* adj, long long m, int n, int* err) {
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (long long)gridDim.x * blockDim.x) {
        int w = adj[e];
        if (w < 0 || w >= n) atomicOr(err, V_RANGE);
    }
}

__global__ void k_perm_keys(const int* off, int n, unsigned long long* keys, int* maxdeg) {
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    unsigned int d = (unsigned int)(off[v + 1] - off[v]);
    keys[v] = ((unsigned long long)(0xFFFFFFFFu - d) << 32) | (unsigned int)v;
    atomicMax(maxdeg, (int)d);
}

__global__ void k_perm_from_keys(const unsigned long long* keys, const int* off, int n, int* perm, int* inv,
                                 int* ndeg) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    int v = (int)(keys[r] & 0xFFFFFFFFull);
    perm[r] = v;
    inv[v] = r;
    ndeg[r] = off[v + 1] - off[v];
}

// one warp per original row: arc keys (inv[row] << 32 | inv[col])
__global__ void k_arc_keys(const int* off, const int* adj, const int* inv, int n, unsigned long long* keys) {
    const int lane = threadIdx.x & 31;
    const long long wg = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long v = wg; v < n; v += nw) {
        const unsigned long long r = (unsigned long long)inv[v] << 32;
        for (long long e = off[v] + lane; e < off[v + 1]; e += 32) keys[e] = r | (unsigned int)inv[adj[e]];
    }
}

__global__ void k_csr_from_keys(const unsigned long long* keys, long long m, int n, int* noff, int* nadj, int* err) {
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (long long)gridDim.x * blockDim.x) {
        const unsigned long long k = keys[e];
        const int r = (int)(k >> 32), c = (int)(k & 0xFFFFFFFFull);
        nadj[e] = c;
        if (r == c) atomicOr(err, V_SELF);
        const int prev = e > 0 ? (int)(keys[e - 1] >> 32) : -1;
        if (e > 0 && keys[e - 1] == k) atomicOr(err, V_DUP);
        for (int rr = prev + 1; rr <= r; ++rr) noff[rr] = (int)e;
        if (e == m - 1)
            for (int rr = r + 1; rr <= n; ++rr) noff[rr] = (int)m;
    }
}

// one warp per relabelled row: reversed arc keys (col << 32 | row) for the in-CSR
__global__ void k_rev_keys(const int* noff, const int* nadj, int n, unsigned long long* keys) {
    const int lane = threadIdx.x & 31;
    const long long wg = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long r = wg; r < n; r += nw)
        for (long long e = noff[r] + lane; e < noff[r + 1]; e += 32)
            keys[e] = ((unsigned long long)(unsigned int)nadj[e] << 32) | (unsigned int)r;
}

__global__ void k_max_row(const int* noff, int n, int* out) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) atomicMax(out, noff[r + 1] - noff[r]);
}

__global__ void k_fill_empty_offsets(int* noff, int n) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r <= n) noff[r] = 0;
}

__global__ void k_check_symmetry(const int* noff, const int* nadj, int n, int* err) {
    const int lane = threadIdx.x & 31;
    const long long wg = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long r = wg; r < n; r += nw) {
        for (long long e = noff[r] + lane; e < noff[r + 1]; e += 32) {
            const int c = nadj[e];
            int lo = noff[c], hi = noff[c + 1];
            while (lo < hi) {
                int mid = (lo + hi) >> 1;
                if (nadj[mid] < r) lo = mid + 1;
                else hi = mid;
            }
            if (lo >= noff[c + 1] || nadj[lo] != (int)r) atomicOr(err, V_ASYM);
        }
    }
}

__global__ void k_count_nz(const int* noff, int n, int* n_nz) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int d = noff[r + 1] - noff[r];
    const int dn = (r + 1 < n) ? noff[r + 2] - noff[r + 1] : 0;
    if (d > 0 && dn == 0) atomicMax(n_nz, r + 1);
}

// ---------------------------------------------------------------- radix sort
__global__ void k_radix_hist(const unsigned long long* keys, long long nkeys, int shift, int nblocks,
                             unsigned int* counts) {
    __shared__ unsigned int h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const long long base = (long long)blockIdx.x * kTile;
    for (int i = 0; i < kSortIPT; ++i) {
        const long long idx = base + (long long)i * kSortThreads + threadIdx.x;
        if (idx < nkeys) atomicAdd(&h[(keys[idx] >> shift) & 0xFF], 1u);
    }
    __syncthreads();
    counts[(size_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

__global__ void k_radix_scatter(const unsigned long long* keys, unsigned long long* out, long long nkeys, int shift,
                                int nblocks, const unsigned long long* goff) {
    __shared__ unsigned int wc[kSortWarps][256];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kSortWarps * 256; i += kSortThreads) (&wc[0][0])[i] = 0;
    __syncthreads();
    // warp-striped tile: warp w owns [w*512, (w+1)*512), round i covers 32 consecutive keys
    const long long base = (long long)blockIdx.x * kTile + (long long)wid * (32 * kSortIPT);
    unsigned long long k[kSortIPT];
    int dig[kSortIPT];
    unsigned int rk[kSortIPT];
    const unsigned int lt = (1u << lane) - 1u;
#pragma unroll
    for (int i = 0; i < kSortIPT; ++i) {
        const long long idx = base + i * 32 + lane;
        const bool ok = idx < nkeys;
        k[i] = ok ? keys[idx] : 0ull;
        dig[i] = ok ? (int)((k[i] >> shift) & 0xFF) : 256;
        const unsigned int peers = __match_any_sync(0xffffffffu, dig[i]);
        const unsigned int before = (ok ? wc[wid][dig[i]] : 0u);
        rk[i] = before + __popc(peers & lt);
        __syncwarp();
        if (ok && (peers & lt) == 0) wc[wid][dig[i]] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    {
        const int d = threadIdx.x;  // 256 threads = 256 digits
        unsigned int run = 0;
        for (int w = 0; w < kSortWarps; ++w) {
            unsigned int t = wc[w][d];
            wc[w][d] = run;
            run += t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kSortIPT; ++i) {
        if (dig[i] < 256) {
            const unsigned long long pos = goff[(size_t)dig[i] * nblocks + blockIdx.x] + wc[wid][dig[i]] + rk[i];
            out[pos] = k[i];
        }
    }
}

// exclusive scan of unsigned counts into 64-bit offsets (block sums + recursion)
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 2048;

__global__ void k_scan_block(const unsigned long long* in32or64, int in_is_u32, unsigned long long* out, long long n,
                             unsigned long long* block_sums) {
    __shared__ unsigned long long s[kScanItems];
    const long long base = (long long)blockIdx.x * kScanItems;
    for (int i = threadIdx.x; i < kScanItems; i += kScanThreads) {
        const long long idx = base + i;
        unsigned long long v = 0;
        if (idx < n)
            v = in_is_u32 ? (unsigned long long)reinterpret_cast<const unsigned int*>(in32or64)[idx] : in32or64[idx];
        s[i] = v;
    }
    __syncthreads();
    // Blelloch scan over kScanItems
    for (int d = 1; d < kScanItems; d <<= 1) {
        for (int i = threadIdx.x; i < kScanItems / (2 * d); i += kScanThreads) {
            const int a = (2 * i + 1) * d - 1, b = (2 * i + 2) * d - 1;
            s[b] += s[a];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (block_sums) block_sums[blockIdx.x] = s[kScanItems - 1];
        s[kScanItems - 1] = 0;
    }
    __syncthreads();
    for (int d = kScanItems / 2; d >= 1; d >>= 1) {
        for (int i = threadIdx.x; i < kScanItems / (2 * d); i += kScanThreads) {
            const int a = (2 * i + 1) * d - 1, b = (2 * i + 2) * d - 1;
            const unsigned long long t = s[a];
            s[a] = s[b];
            s[b] += t;
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < kScanItems; i += kScanThreads) {
        const long long idx = base + i;
        if (idx < n) out[idx] = s[i];
    }
}

__global__ void k_scan_add(unsigned long long* out, long long n, const unsigned long long* block_offs) {
    const long long idx = (long long)blockIdx.x * kScanItems;
    for (int i = threadIdx.x; i < kScanItems; i += kScanThreads)
        if (idx + i < n) out[idx + i] += block_offs[blockIdx.x];
}

struct Pool {
    AllocFn alloc;
    FreeFn dfree;
    cudaStream_t st;
    bool oom = false;
    void* get(size_t b) {
        void* p = alloc(b ? b : 16, st);
        if (!p) oom = true;
        return p;
    }
    void put(void* p) {
        if (p) dfree(p, st);
    }
};

// exclusive scan of n values (u32 input when in_is_u32) into out (u64)
cudaError_t scan_u64(Pool& pool, const void* in, int in_is_u32, unsigned long long* out, long long n) {
    if (n <= 0) return cudaSuccess;
    const long long nb = (n + kScanItems - 1) / kScanItems;
    unsigned long long* sums = nullptr;
    unsigned long long* sums_scanned = nullptr;
    if (nb > 1) {
        sums = (unsigned long long*)pool.get(sizeof(unsigned long long) * nb);
        sums_scanned = (unsigned long long*)pool.get(sizeof(unsigned long long) * nb);
        if (pool.oom) { pool.put(sums); pool.put(sums_scanned); return cudaErrorMemoryAllocation; }
    }
    k_scan_block<<<(unsigned)nb, kScanThreads, 0, pool.st>>>((const unsigned long long*)in, in_is_u32, out, n, sums);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && nb > 1) {
        e = scan_u64(pool, sums, 0, sums_scanned, nb);
        if (e == cudaSuccess) {
            k_scan_add<<<(unsigned)nb, kScanThreads, 0, pool.st>>>(out, n, sums_scanned);
            e = cudaGetLastError();
        }
    }
    pool.put(sums);
    pool.put(sums_scanned);
    return e;
}

// Sort keys[0..nkeys) by the 8-bit digits at the given shifts (least significant first).
// Result ends in *keys (the two buffers may be swapped).
cudaError_t radix_sort(Pool& pool, unsigned long long** keys, unsigned long long** tmp, long long nkeys,
                       const int* shifts, int npass) {
    if (nkeys <= 1 || npass == 0) return cudaSuccess;
    const long long nb = (nkeys + kTile - 1) / kTile;
    if (nb > (1ll << 31) / 256) return cudaErrorInvalidValue;
    unsigned int* counts = (unsigned int*)pool.get(sizeof(unsigned int) * 256 * nb);
    unsigned long long* goff = (unsigned long long*)pool.get(sizeof(unsigned long long) * 256 * nb);
    if (pool.oom) { pool.put(counts); pool.put(goff); return cudaErrorMemoryAllocation; }
    cudaError_t e = cudaSuccess;
    for (int ps = 0; ps < npass && e == cudaSuccess; ++ps) {
        k_radix_hist<<<(unsigned)nb, kSortThreads, 0, pool.st>>>(*keys, nkeys, shifts[ps], (int)nb, counts);
        e = cudaGetLastError();
        if (e != cudaSuccess) break;
        e = scan_u64(pool, counts, 1, goff, 256 * nb);
        if (e != cudaSuccess) break;
        k_radix_scatter<<<(unsigned)nb, kSortThreads, 0, pool.st>>>(*keys, *tmp, nkeys, shifts[ps], (int)nb, goff);
        e = cudaGetLastError();
        unsigned long long* t = *keys;
        *keys = *tmp;
        *tmp = t;
    }
    pool.put(counts);
    pool.put(goff);
    return e;
}

int bits_for(unsigned long long x) {
    int b = 0;
    while (b < 64 && (x >> b) != 0) ++b;
    return b;
}

}  // namespace

cudaError_t ingest(const int* d_off, const int* d_adj, int n, long long m, bool validate, bool directed,
                   cudaStream_t st, AllocFn alloc, FreeFn dfree, IngestOut* out, bool* oom) {
    Pool pool{alloc, dfree, st};
    out->reason = 0;
    out->off = nullptr; out->adj = nullptr; out->perm = nullptr; out->inv = nullptr;
    out->ioff = nullptr; out->iadj = nullptr; out->max_in_deg = 0;
    out->max_deg = 0; out->n_nz = 0;
    *oom = false;
    int* d_err = (int*)pool.get(sizeof(int) * 5);
    if (pool.oom) { *oom = true; return cudaErrorMemoryAllocation; }
    int h_err[4] = {0, 0, 0, 0};
    cudaError_t e = cudaMemsetAsync(d_err, 0, sizeof(int) * 5, st);
    auto fail = [&](cudaError_t ee) { *oom = pool.oom; return ee; };

    // 1. offsets and index range (always: later kernels index with these values)
    if (n > 0) {
        k_check_offsets<<<(n + 255) / 256, 256, 0, st>>>(d_off, n, m, d_err);
        if (m > 0) k_check_range<<<1184, 256, 0, st>>>(d_adj, m, n, d_err);
    } else {
        k_check_offsets<<<1, 1, 0, st>>>(d_off, 0, m, d_err);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(e);
    if ((e = cudaMemcpyAsync(h_err, d_err, sizeof(int) * 2, cudaMemcpyDeviceToHost, st)) != cudaSuccess) return fail(e);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return fail(e);
    if (h_err[0] & V_OFFSETS) { out->reason = 1; pool.put(d_err); return cudaSuccess; }
    if (h_err[0] & V_RANGE) { out->reason = 2; pool.put(d_err); return cudaSuccess; }

    out->off = (int*)pool.get(sizeof(int) * ((size_t)n + 1));
    out->adj = (int*)pool.get(sizeof(int) * (size_t)(m > 0 ? m : 1));
    out->perm = (int*)pool.get(sizeof(int) * (size_t)(n > 0 ? n : 1));
    out->inv = (int*)pool.get(sizeof(int) * (size_t)(n > 0 ? n : 1));
    int* ndeg = (int*)pool.get(sizeof(int) * (size_t)(n > 0 ? n : 1));
    const long long nk = (n > m ? n : m) > 0 ? (n > m ? n : m) : 1;
    unsigned long long* ka = (unsigned long long*)pool.get(sizeof(unsigned long long) * (size_t)nk);
    unsigned long long* kb = (unsigned long long*)pool.get(sizeof(unsigned long long) * (size_t)nk);
    auto cleanup_tmp = [&]() { pool.put(ndeg); pool.put(ka); pool.put(kb); pool.put(d_err); };
    if (pool.oom) { cleanup_tmp(); *oom = true; return cudaErrorMemoryAllocation; }

    if (n == 0) {
        k_fill_empty_offsets<<<1, 32, 0, st>>>(out->off, 0);
        e = cudaStreamSynchronize(st);
        cleanup_tmp();
        return fail(e);
    }
    // 2. permutation
    k_perm_keys<<<(n + 255) / 256, 256, 0, st>>>(d_off, n, ka, d_err + 2);
    if ((e = cudaMemcpyAsync(&h_err[2], d_err + 2, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess) {
        cleanup_tmp();
        return fail(e);
    }
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) { cleanup_tmp(); return fail(e); }
    out->max_deg = h_err[2];
    {
        const int b = bits_for((unsigned long long)out->max_deg);
        int shifts[8], np = 0;
        for (int s = 0; s < b; s += 8) shifts[np++] = 32 + s;
        if ((e = radix_sort(pool, &ka, &kb, n, shifts, np)) != cudaSuccess) { cleanup_tmp(); return fail(e); }
    }
    k_perm_from_keys<<<(n + 255) / 256, 256, 0, st>>>(ka, d_off, n, out->perm, out->inv, ndeg);
    // 3. arcs
    if (m > 0) {
        k_arc_keys<<<1184, 256, 0, st>>>(d_off, d_adj, out->inv, n, ka);
        const int b = bits_for((unsigned long long)(n - 1));
        int shifts[16], np = 0;
        for (int s = 0; s < b; s += 8) shifts[np++] = s;
        for (int s = 0; s < b; s += 8) shifts[np++] = 32 + s;
        if ((e = radix_sort(pool, &ka, &kb, m, shifts, np)) != cudaSuccess) { cleanup_tmp(); return fail(e); }
        k_csr_from_keys<<<1184, 256, 0, st>>>(ka, m, n, out->off, out->adj, d_err);
        if (validate && !directed) k_check_symmetry<<<1184, 256, 0, st>>>(out->off, out->adj, n, d_err);
    } else {
        k_fill_empty_offsets<<<(n + 1 + 255) / 256, 256, 0, st>>>(out->off, n);
    }
    if (directed) {
        // in-CSR (the transpose, rows sorted) for the pull steps of directed graphs;
        // its duplicate/self-loop flags go to a slot nobody reads (the out-CSR's count)
        out->ioff = (int*)pool.get(sizeof(int) * ((size_t)n + 1));
        out->iadj = (int*)pool.get(sizeof(int) * (size_t)(m > 0 ? m : 1));
        if (pool.oom) { cleanup_tmp(); *oom = true; return cudaErrorMemoryAllocation; }
        if (m > 0) {
            k_rev_keys<<<1184, 256, 0, st>>>(out->off, out->adj, n, ka);
            const int b = bits_for((unsigned long long)(n - 1));
            int shifts[16], np = 0;
            for (int s = 0; s < b; s += 8) shifts[np++] = s;
            for (int s = 0; s < b; s += 8) shifts[np++] = 32 + s;
            if ((e = radix_sort(pool, &ka, &kb, m, shifts, np)) != cudaSuccess) { cleanup_tmp(); return fail(e); }
            k_csr_from_keys<<<1184, 256, 0, st>>>(ka, m, n, out->ioff, out->iadj, d_err + 4);
        } else {
            k_fill_empty_offsets<<<(n + 1 + 255) / 256, 256, 0, st>>>(out->ioff, n);
        }
        cudaMemsetAsync(d_err + 4, 0, sizeof(int), st);
        k_max_row<<<(n + 255) / 256, 256, 0, st>>>(out->ioff, n, d_err + 4);
        int h_in = 0;
        if ((e = cudaMemcpyAsync(&h_in, d_err + 4, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess) {
            cleanup_tmp();
            return fail(e);
        }
        out->max_in_deg = h_in;
    }
    cudaMemsetAsync(d_err + 3, 0, sizeof(int), st);
    k_count_nz<<<(n + 255) / 256, 256, 0, st>>>(out->off, n, d_err + 3);
    if ((e = cudaGetLastError()) != cudaSuccess) { cleanup_tmp(); return fail(e); }
    if ((e = cudaMemcpyAsync(h_err, d_err, sizeof(int) * 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess) {
        cleanup_tmp();
        return fail(e);
    }
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) { cleanup_tmp(); return fail(e); }
    out->n_nz = h_err[3];
    if (validate) {
        if (h_err[0] & V_SELF) out->reason = 3;
        else if (h_err[0] & V_DUP) out->reason = 4;
        else if (h_err[0] & V_ASYM) out->reason = 5;
    }
    cleanup_tmp();
    return cudaSuccess;
}

}  // namespace bcx
