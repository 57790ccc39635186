// Initial states, lattice validation and the integer observables of Section 7.
#include <algorithm>

#include <cuda_runtime.h>

#include "fskmc_internal.h"
#include "philox.cuh"

namespace fskmc {

namespace {

// Site i of replica rep is 1 iff word 0 of Philox(seed, (i,0,0,rep|2<<24)) < p 2^32.
__global__ void init_bernoulli_kernel(uint8_t *lat, int64_t n, uint64_t seed, double thr,
                                      uint32_t rep)
{
    const uint32_t c3 = rep | (TAG_INIT << 24);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        u32x4 o = draw(seed, (uint32_t)i, 0u, 0u, c3);
        lat[i] = __uint2double_rn(o.x) < thr ? 1 : 0;
    }
}

// Gaussian bump: species with probability (amp * gx[x]) * gy[y].
__global__ void init_bump_kernel(uint8_t *lat, int lx, int ly, uint64_t seed,
                                 const double *gx, const double *gy, double amp, int species,
                                 uint32_t rep)
{
    const uint32_t c3 = rep | (TAG_INIT << 24);
    const int64_t n = (int64_t)lx * ly;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int x = (int)(i % lx), y = (int)(i / lx);
        u32x4 o = draw(seed, (uint32_t)i, 0u, 0u, c3);
        double p = __dmul_rn(__dmul_rn(amp, gx[x]), gy[y]);
        lat[i] = __uint2double_rn(o.x) < __dmul_rn(p, 4294967296.0) ? (uint8_t)species : 0;
    }
}

__global__ void validate_kernel(const uint8_t *lat, int64_t n, int nstates, unsigned int *bad)
{
    unsigned int c = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        c += lat[i] >= nstates;
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(bad, c);
}

__global__ void pack_kernel(const uint8_t *bytes, uint32_t *words, int64_t nwords)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nwords;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint8_t *b = bytes + 32 * i;
        uint32_t w = 0;
#pragma unroll
        for (int k = 0; k < 32; ++k) w |= (uint32_t)(b[k] & 1u) << k;
        words[i] = w;
    }
}

__global__ void unpack_kernel(const uint32_t *words, uint8_t *bytes, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        bytes[i] = (uint8_t)((words[i >> 5] >> (i & 31)) & 1u);
}

// Site (x, y) of a row-major lattice, one byte per site or bit-packed.
template <bool PACKED>
__device__ __forceinline__ int site_at(const uint8_t *lat, int lx, int y, int x)
{
    if (PACKED) {
        const uint32_t *w = reinterpret_cast<const uint32_t *>(lat);
        return (int)((w[(int64_t)y * (lx >> 5) + (x >> 5)] >> (x & 31)) & 1u);
    }
    return lat[(int64_t)y * lx + x];
}

// Row chunks of OBS_CHUNK sites, one per block (grid-stride over the rows'
// chunks). Accumulators in shared memory as 32-bit per block, flushed with
// 64-bit atomics. A ring (ly == 1) has no vertical bonds: its vertical pairs
// and G_y are 0.
constexpr int OBS_CHUNK = 4096;

template <bool PACKED>
__global__ void observables_kernel(const uint8_t *lat, int lx, int ly, int rmax,
                                   unsigned long long *out)
{
    extern __shared__ unsigned int acc[];  // 4 + 2*rmax
    const int nacc = 4 + 2 * rmax;
    for (int i = threadIdx.x; i < nacc; i += blockDim.x) acc[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const bool vert = ly > 1;
    const int nch = (lx + OBS_CHUNK - 1) / OBS_CHUNK;
    for (int64_t task = blockIdx.x; task < (int64_t)ly * nch; task += gridDim.x) {
        const int y = (int)(task / nch);
        const int xa = (int)(task % nch) * OBS_CHUNK;
        const int xb = min(lx, xa + OBS_CHUNK);
        const int yd = (y + 1) % ly;
        // counts and nearest-neighbour pairs; the tail is handled by the
        // predicate, so every lane reaches the reduces
        for (int x0 = xa; x0 < xb; x0 += blockDim.x) {
            int x = x0 + threadIdx.x;
            unsigned int c0 = 0, c1 = 0, c2 = 0, pr = 0;
            const int s = x < xb ? site_at<PACKED>(lat, lx, y, x) : -1;
            if (x < xb) {
                c0 = s == 0; c1 = s == 1; c2 = s == 2;
                if (s == 1) pr = (site_at<PACKED>(lat, lx, y, (x + 1) % lx) == 1) +
                                 (vert && site_at<PACKED>(lat, lx, yd, x) == 1);
            }
            c0 = __reduce_add_sync(0xffffffffu, c0);
            c1 = __reduce_add_sync(0xffffffffu, c1);
            c2 = __reduce_add_sync(0xffffffffu, c2);
            pr = __reduce_add_sync(0xffffffffu, pr);
            if (lane == 0) {
                atomicAdd(&acc[0], c0); atomicAdd(&acc[1], c1);
                atomicAdd(&acc[2], c2); atomicAdd(&acc[3], pr);
            }
            for (int r = 1; r <= rmax; ++r) {
                unsigned int gxv = 0, gyv = 0;
                if (s == 1) {
                    gxv = site_at<PACKED>(lat, lx, y, (x + r) % lx) == 1;
                    gyv = vert && site_at<PACKED>(lat, lx, (y + r) % ly, x) == 1;
                }
                gxv = __reduce_add_sync(0xffffffffu, gxv);
                gyv = __reduce_add_sync(0xffffffffu, gyv);
                if (lane == 0) {
                    if (gxv) atomicAdd(&acc[4 + r - 1], gxv);
                    if (gyv) atomicAdd(&acc[4 + rmax + r - 1], gyv);
                }
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nacc; i += blockDim.x)
        if (acc[i]) atomicAdd(&out[i], (unsigned long long)acc[i]);
}

// Issue-order buckets of a cell's event count W: exact below 64, then 8
// buckets per power of two (descending bucket = heavier).
__device__ __forceinline__ int order_bucket(int32_t W)
{
    if (W < 64) return W < 0 ? 0 : W;
    const int e = 31 - __clz(W);  // 6..30
    return 64 + (e - 6) * 8 + ((W >> (e - 3)) & 7);
}

constexpr int ORDER_CHUNK = 4096;  // active cells per block
constexpr int ORDER_THREADS = 512;

// The u-th active cell of colour col in row-major order.
__device__ __forceinline__ int active_cell(const Replica &R, int col, int u)
{
    const int half = R.ncx >> 1;
    const int cy = u / half;
    return cy * R.ncx + 2 * (u - cy * half) + ((col + cy) & 1);
}

// Block-local histogram of the buckets of this block's chunk of active cells.
__device__ void order_local_hist(const Replica &R, int col, int u0, int n, const int32_t *wl,
                                 int32_t *h)
{
    for (int i = threadIdx.x; i < ORDER_BUCKETS; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const int u1 = min(n, u0 + ORDER_CHUNK);
    for (int u = u0 + threadIdx.x; u < u1; u += blockDim.x)
        atomicAdd(&h[order_bucket(wl[R.cell_off + active_cell(R, col, u)])], 1);
    __syncthreads();
}

__global__ void order_hist_kernel(const Replica *reps, int r0, int c0, const int32_t *wl,
                                  int32_t *hist)
{
    __shared__ int32_t h[ORDER_BUCKETS];
    const Replica &R = reps[r0 + blockIdx.y];
    const int col = c0 + blockIdx.z;
    const int n = (R.ncx >> 1) * R.ncy;
    const int u0 = blockIdx.x * ORDER_CHUNK;
    if (u0 >= n) return;  // uniform over the block
    order_local_hist(R, col, u0, n, wl, h);
    int32_t *gh = hist + ((size_t)blockIdx.y * 2 + blockIdx.z) * ORDER_BUCKETS;
    for (int i = threadIdx.x; i < ORDER_BUCKETS; i += blockDim.x)
        if (h[i]) atomicAdd(&gh[i], h[i]);
}

__global__ void order_scatter_kernel(const Replica *reps, int r0, int c0, const int32_t *wl,
                                     const int32_t *hist, int32_t *cursor, int32_t *order)
{
    __shared__ int32_t h[ORDER_BUCKETS], base[ORDER_BUCKETS];
    const Replica &R = reps[r0 + blockIdx.y];
    const int col = c0 + blockIdx.z;
    const int n = (R.ncx >> 1) * R.ncy;
    const int u0 = blockIdx.x * ORDER_CHUNK;
    if (u0 >= n) return;
    order_local_hist(R, col, u0, n, wl, h);
    const size_t seg = ((size_t)blockIdx.y * 2 + blockIdx.z) * ORDER_BUCKETS;
    // bucket b starts after every heavier bucket: exclusive scan in
    // descending bucket order, 9 buckets per lane of warp 0
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        int v[9], sum = 0;
#pragma unroll
        for (int t = 0; t < 9; ++t) {
            const int d = lane * 9 + t, b = ORDER_BUCKETS - 1 - d;
            v[t] = d < ORDER_BUCKETS ? hist[seg + b] : 0;
            sum += v[t];
        }
        int incl = sum;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int x = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += x;
        }
        int acc = incl - sum;
#pragma unroll
        for (int t = 0; t < 9; ++t) {
            const int d = lane * 9 + t;
            if (d < ORDER_BUCKETS) base[ORDER_BUCKETS - 1 - d] = acc;
            acc += v[t];
        }
    }
    __syncthreads();
    // reserve this block's range in every bucket it uses
    for (int i = threadIdx.x; i < ORDER_BUCKETS; i += blockDim.x)
        if (h[i]) base[i] += atomicAdd(&cursor[seg + i], h[i]);
    __syncthreads();
    int32_t *out = order + R.cell_off + (size_t)col * n;
    const int u1 = min(n, u0 + ORDER_CHUNK);
    for (int u = u0 + threadIdx.x; u < u1; u += blockDim.x) {
        const int m = active_cell(R, col, u);
        out[atomicAdd(&base[order_bucket(wl[R.cell_off + m])], 1)] = m;
    }
}

// Whole issue list of one (replica, colour) in one block, for windows of at
// most ORDER_SINGLE active cells: histogram, scan and scatter in shared
// memory, no global scratch.
constexpr int ORDER_SINGLE = 32768;

__global__ void order_single_kernel(const Replica *reps, int r0, int c0, const int32_t *wl,
                                    int32_t *order)
{
    __shared__ int32_t h[ORDER_BUCKETS], base[ORDER_BUCKETS];
    const Replica &R = reps[r0 + blockIdx.x];
    const int col = c0 + blockIdx.y;
    const int n = (R.ncx >> 1) * R.ncy;
    for (int i = threadIdx.x; i < ORDER_BUCKETS; i += blockDim.x) h[i] = 0;
    __syncthreads();
    for (int u = threadIdx.x; u < n; u += blockDim.x)
        atomicAdd(&h[order_bucket(wl[R.cell_off + active_cell(R, col, u)])], 1);
    __syncthreads();
    if (threadIdx.x < 32) {  // exclusive scan, heaviest bucket first
        const int lane = threadIdx.x;
        int v[9], sum = 0;
#pragma unroll
        for (int t = 0; t < 9; ++t) {
            const int d = lane * 9 + t;
            v[t] = d < ORDER_BUCKETS ? h[ORDER_BUCKETS - 1 - d] : 0;
            sum += v[t];
        }
        int incl = sum;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int x = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += x;
        }
        int acc = incl - sum;
#pragma unroll
        for (int t = 0; t < 9; ++t) {
            const int d = lane * 9 + t;
            if (d < ORDER_BUCKETS) base[ORDER_BUCKETS - 1 - d] = acc;
            acc += v[t];
        }
    }
    __syncthreads();
    int32_t *out = order + R.cell_off + (size_t)col * n;
    for (int u = threadIdx.x; u < n; u += blockDim.x) {
        const int m = active_cell(R, col, u);
        out[atomicAdd(&base[order_bucket(wl[R.cell_off + m])], 1)] = m;
    }
}

int grid_for(int64_t n, int block)
{
    int64_t b = (n + block - 1) / block;
    if (b > 152 * 32) b = 152 * 32;
    return b < 1 ? 1 : (int)b;
}

}  // namespace

cudaError_t launch_init_bernoulli(uint8_t *lat, int lx, int ly, uint64_t seed, double p,
                                  uint32_t rep, cudaStream_t s)
{
    int64_t n = (int64_t)lx * ly;
    init_bernoulli_kernel<<<grid_for(n, 256), 256, 0, s>>>(lat, n, seed, p * 4294967296.0, rep);
    return cudaGetLastError();
}

cudaError_t launch_init_bump(uint8_t *lat, int lx, int ly, uint64_t seed, const double *gx,
                             const double *gy, double amp, int species, uint32_t rep,
                             cudaStream_t s)
{
    int64_t n = (int64_t)lx * ly;
    init_bump_kernel<<<grid_for(n, 256), 256, 0, s>>>(lat, lx, ly, seed, gx, gy, amp, species,
                                                      rep);
    return cudaGetLastError();
}

cudaError_t launch_validate(const uint8_t *lat, int64_t n, int nstates, unsigned int *bad,
                            cudaStream_t s)
{
    validate_kernel<<<grid_for(n, 256), 256, 0, s>>>(lat, n, nstates, bad);
    return cudaGetLastError();
}

// Word-parallel observables for lattices whose rows are whole 32-site words
// (lx % 32 == 0, rows 16-byte aligned) and r <= 32: the indicator of state
// 1 is packed 32 sites per word (bit t of word c of row y = site
// (32c + t, y)), and every sum becomes popcounts of ANDs of words --
//   pairs   = sum popc(w & (w >> 1 | next << 31)) + popc(w & below)
//   G_x(r)  = sum popc(w & funnel(w, next, r)),   G_y(r) = sum popc(w & w[y + r])
// (next: the word to the right, below / w[y + r]: the same column r rows
// down, both periodic). A block stages the indicator words of OBS_TY rows
// and OBS_CW word columns, plus r_max rows below and one column to the right,
// in shared memory; the byte lattice is read once with 16-byte loads
// (plus r_max / OBS_TY of it again for the rows below). Exact integer sums,
// equal to the site-by-site kernel's.
constexpr int OBS_TY = 32, OBS_CW = 32, OBS_RMAX_WORDS = 32;

// Bytes v (4 sites) -> 4 indicator bits of state `st` at bits 0..3, by a
// bytewise compare and one multiply that gathers the compare's top bits.
__device__ __forceinline__ uint32_t nibble_eq(uint32_t v, uint32_t st4)
{
    const uint32_t t = (__vcmpeq4(v, st4) & 0x80808080u) >> 7;  // bits 0, 8, 16, 24
    return (t * 0x00204081u) >> 21 & 0xFu;
}

template <bool PACKED>
__global__ void __launch_bounds__(256) observables_words_kernel(const uint8_t *lat, int lx, int ly,
                                                                 int rmax, unsigned long long *out)
{
    __shared__ uint32_t S[(OBS_TY + OBS_RMAX_WORDS) * (OBS_CW + 1)];
    __shared__ unsigned int acc[4 + 2 * OBS_RMAX_WORDS];
    const int nacc = 4 + 2 * rmax;
    for (int i = threadIdx.x; i < nacc; i += blockDim.x) acc[i] = 0;
    const bool vert = ly > 1;
    const int nw = lx >> 5;
    const int c0 = blockIdx.x * OBS_CW, y0 = blockIdx.y * OBS_TY;
    const int cw = min(OBS_CW, nw - c0), ty = min(OBS_TY, ly - y0);
    const int rows = ty + (vert ? max(rmax, 1) : 0);  // the rows below: G_y and the vertical pairs
    const int SW = OBS_CW + 1;
    // stage the indicator words (rows and columns periodic); count states
    // 1 and 2 in this tile's own words
    unsigned int n1 = 0, n2 = 0;
    for (int i = threadIdx.x; i < rows * (cw + 1); i += blockDim.x) {
        const int r = i / (cw + 1), c = i - r * (cw + 1);
        int gy = y0 + r;
        while (gy >= ly) gy -= ly;
        int gc = c0 + c;
        if (gc >= nw) gc -= nw;
        uint32_t word, w2 = 0u;
        if (PACKED) {
            word = reinterpret_cast<const uint32_t *>(lat)[(int64_t)gy * nw + gc];
        } else {
            const uint4 *p = reinterpret_cast<const uint4 *>(lat + (int64_t)gy * lx + 32 * gc);
            const uint4 a = p[0], b = p[1];
            const uint32_t v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
            word = 0u;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                word |= nibble_eq(v[k], 0x01010101u) << (4 * k);
                w2 |= nibble_eq(v[k], 0x02020202u) << (4 * k);
            }
        }
        S[r * SW + c] = word;
        if (r < ty && c < cw) {
            n1 += __popc(word);
            n2 += __popc(w2);
        }
    }
    __syncthreads();
    unsigned int pr = 0;
    unsigned int gx[OBS_RMAX_WORDS], gy[OBS_RMAX_WORDS];
#pragma unroll
    for (int r = 0; r < OBS_RMAX_WORDS; ++r) gx[r] = gy[r] = 0u;
    for (int i = threadIdx.x; i < ty * cw; i += blockDim.x) {
        const int r = i / cw, c = i - r * cw;
        const uint32_t w = S[r * SW + c], nx = S[r * SW + c + 1];
        pr += __popc(w & __funnelshift_r(w, nx, 1));
        if (vert) pr += __popc(w & S[(r + 1) * SW + c]);
#pragma unroll
        for (int d = 1; d <= OBS_RMAX_WORDS; ++d) {
            if (d > rmax) break;
            gx[d - 1] += __popc(w & __funnelshift_rc(w, nx, d));
            if (vert) gy[d - 1] += __popc(w & S[(r + d) * SW + c]);
        }
    }
    // block sums: warp reduce, then shared atomics
    const int lane = threadIdx.x & 31;
    const unsigned int ncell = (unsigned int)(ty * cw) * 32u;
    {
        const unsigned int a1 = __reduce_add_sync(0xffffffffu, n1);
        const unsigned int a2 = __reduce_add_sync(0xffffffffu, n2);
        const unsigned int ap = __reduce_add_sync(0xffffffffu, pr);
        if (lane == 0) { atomicAdd(&acc[1], a1); atomicAdd(&acc[2], a2); atomicAdd(&acc[3], ap); }
    }
#pragma unroll
    for (int d = 0; d < OBS_RMAX_WORDS; ++d) {
        if (d >= rmax) break;
        const unsigned int a = __reduce_add_sync(0xffffffffu, gx[d]);
        const unsigned int b = __reduce_add_sync(0xffffffffu, gy[d]);
        if (lane == 0) {
            if (a) atomicAdd(&acc[4 + d], a);
            if (b) atomicAdd(&acc[4 + rmax + d], b);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) acc[0] = ncell - acc[1] - acc[2];
    __syncthreads();
    for (int i = threadIdx.x; i < nacc; i += blockDim.x)
        if (acc[i]) atomicAdd(&out[i], (unsigned long long)acc[i]);
}

cudaError_t launch_observables(const uint8_t *lat, int lx, int ly, int rmax,
                               unsigned long long *out, cudaStream_t s, bool packed)
{
    const bool words = (lx & 31) == 0 && rmax <= OBS_RMAX_WORDS &&
                       (reinterpret_cast<uintptr_t>(lat) & 15u) == 0;
    if (words) {
        const dim3 grid((unsigned)((lx / 32 + OBS_CW - 1) / OBS_CW), (unsigned)((ly + OBS_TY - 1) / OBS_TY));
        if (packed) observables_words_kernel<true><<<grid, 256, 0, s>>>(lat, lx, ly, rmax, out);
        else observables_words_kernel<false><<<grid, 256, 0, s>>>(lat, lx, ly, rmax, out);
        return cudaGetLastError();
    }
    const int64_t tasks = (int64_t)ly * ((lx + OBS_CHUNK - 1) / OBS_CHUNK);
    const int grid = tasks < 152 * 8 ? (int)tasks : 152 * 8;
    size_t smem = sizeof(unsigned int) * (size_t)(4 + 2 * rmax);
    if (packed) observables_kernel<true><<<grid, 256, smem, s>>>(lat, lx, ly, rmax, out);
    else observables_kernel<false><<<grid, 256, smem, s>>>(lat, lx, ly, rmax, out);
    return cudaGetLastError();
}

cudaError_t launch_order(const Replica *reps_host, const Replica *reps_dev, int r0, int nrep,
                         int c0, int c1, int qx, int qy, const int32_t *workload, int32_t *order,
                         int32_t *hist, int32_t *cursor, cudaStream_t s)
{
    (void)qx;
    (void)qy;
    if (nrep < 1 || nrep > 65535 || c0 < 0 || c1 > 1 || c0 > c1) return cudaErrorInvalidValue;
    int64_t most = 0;
    for (int r = r0; r < r0 + nrep; ++r)
        most = std::max<int64_t>(most, (int64_t)(reps_host[r].ncx / 2) * reps_host[r].ncy);
    if (most == 0) return cudaSuccess;
    if (most <= ORDER_SINGLE) {
        order_single_kernel<<<dim3((unsigned)nrep, (unsigned)(c1 - c0 + 1)), 1024, 0, s>>>(
            reps_dev, r0, c0, workload, order);
        return cudaGetLastError();
    }
    const size_t words = (size_t)nrep * 2 * ORDER_BUCKETS;
    cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(int32_t) * words, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(cursor, 0, sizeof(int32_t) * words, s);
    if (e != cudaSuccess) return e;
    const dim3 grid((unsigned)((most + ORDER_CHUNK - 1) / ORDER_CHUNK), (unsigned)nrep,
                    (unsigned)(c1 - c0 + 1));
    order_hist_kernel<<<grid, ORDER_THREADS, 0, s>>>(reps_dev, r0, c0, workload, hist);
    order_scatter_kernel<<<grid, ORDER_THREADS, 0, s>>>(reps_dev, r0, c0, workload, hist, cursor,
                                                        order);
    return cudaGetLastError();
}

cudaError_t launch_pack(const uint8_t *bytes, uint32_t *words, int lx, int ly, cudaStream_t s)
{
    const int64_t nw = (int64_t)(lx >> 5) * ly;
    pack_kernel<<<grid_for(nw, 256), 256, 0, s>>>(bytes, words, nw);
    return cudaGetLastError();
}

cudaError_t launch_unpack(const uint32_t *words, uint8_t *bytes, int lx, int ly, cudaStream_t s)
{
    const int64_t n = (int64_t)lx * ly;
    unpack_kernel<<<grid_for(n, 256), 256, 0, s>>>(words, bytes, n);
    return cudaGetLastError();
}

}  // namespace fskmc
