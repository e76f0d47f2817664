// sf_multiframe.cu -- kernels of multiframe simulation (Sec. IV): COALESCE(F)
// turns candidate pairs of one frame into elements of new frames, and frames
// with equal stabilizer matrices are merged.  Frames of a multiframe have one
// word per phase vector (n <= 63).
//   k_mf_pair    Step 1 of COALESCE: sort the phase vectors so that candidate
//                pairs are neighbours, test each neighbour pair, walk the
//                sorted list once and emit the pairs and the unpaired elements
//   k_mf_gather  copy chosen elements of a frame (scaled) into another buffer
//                or another frame with the same tableau
//   k_mf_import  append exported (canonical) elements of one frame to a frame
//                with the same stabilizer matrix, in the latter's own
//                destabilizer convention (the merge of frames)
#include <algorithm>

#include "sf_canon.cuh"
#include "sf_multiframe.cuh"

namespace {

constexpr int kPairThreads = 1024;
constexpr int kCopyThreads = 256;

// bits of s on the rows of `mask`, row 0 most significant
__device__ __forceinline__ uint64_t row_bits(uint64_t s, uint64_t mask, int n) {
    uint64_t k = 0;
    for (int r = 0; r < n; r++)
        if ((mask >> r) & 1ull) k = (k << 1) | ((s >> r) & 1ull);
    return k;
}

// i^d * a
__device__ __forceinline__ double2 ipow_times(double2 a, int d) {
    switch (d & 3) {
        case 0: return a;
        case 1: return make_double2(-a.y, a.x);
        case 2: return make_double2(-a.x, -a.y);
        default: return make_double2(a.y, -a.x);
    }
}

// One CTA.  Reads the frame's phase vectors from buffer `buf` and their
// canonical amplitudes from the export in buffer `stage` (same order).
// Z_k-rows (no X part, one Z literal) are found on the RREF tableau; the sort
// key is (entries on the other rows, entries on the Z_k-rows), each read with
// row 0 most significant, a bijection of sigma into n <= 63 bits.  Neighbours
// i, i+1 of the sorted list are candidates when they differ only on Z_k-rows
// and a_r = i^d a_j; sigma_j is the member whose entry on the row of the
// smallest differing qubit is 0.  Thread 0 then walks the list from the front
// (a candidate pair takes both neighbours), writing pairs in list order and
// the unpaired elements after them.
// pcap: the power of two the dynamic shared memory was sized for.
__global__ void __launch_bounds__(kPairThreads) k_mf_pair(SfDev d, int buf, int stage, double tol, unsigned pcap,
                                                          MfPair* pairs, uint32_t* keep, uint32_t* counts) {
    extern __shared__ uint64_t sm[];
    __shared__ unsigned long long zmask_s;
    __shared__ int rowq[64];
    const int n = d.n;
    const unsigned long long k = d.kcnt[buf];
    if (*d.status) return;
    if (k > SF_MF_MAXK) {
        if (threadIdx.x == 0) set_status(d.status, SF_ST_CAPACITY, buf);
        return;
    }
    unsigned P = 2;
    while (P < k) P <<= 1;
    if (P > pcap) {  // the count changed since the launch was sized
        if (threadIdx.x == 0) set_status(d.status, SF_ST_INTERNAL, buf, 40u);
        return;
    }
    uint64_t* key = sm;
    uint32_t* ord = reinterpret_cast<uint32_t*>(sm + P);
    uint8_t* flag = reinterpret_cast<uint8_t*>(ord + P);
    if (threadIdx.x == 0) zmask_s = 0ull;
    __syncthreads();
    if (threadIdx.x < 64) {
        int q = 64;
        if ((int)threadIdx.x < n) {
            const uint64_t x = d.mx[threadIdx.x], z = d.mz[threadIdx.x];
            if (x == 0ull && z != 0ull && (z & (z - 1ull)) == 0ull) {
                q = __ffsll((long long)z) - 1;
                atomicOr(&zmask_s, 1ull << threadIdx.x);
            }
        }
        rowq[threadIdx.x] = q;
    }
    __syncthreads();
    const uint64_t zm = zmask_s;
    const uint64_t rows = n == 64 ? ~0ull : ((1ull << n) - 1ull);
    const int nz = __popcll(zm);
    const uint64_t* S = d.sig[buf];
    const double2* A = d.amp[stage];
    for (unsigned i = threadIdx.x; i < P; i += blockDim.x) {
        if (i < k) {
            const uint64_t s = S[i];
            key[i] = (row_bits(s, rows & ~zm, n) << nz) | row_bits(s, zm, n);
            ord[i] = i;
        } else {
            key[i] = ~0ull;
            ord[i] = 0xffffffffu;
        }
    }
    __syncthreads();
    // bitonic sort of (key, ord), ascending; keys of distinct phase vectors differ
    for (unsigned size = 2; size <= P; size <<= 1) {
        for (unsigned stride = size >> 1; stride > 0; stride >>= 1) {
            for (unsigned i = threadIdx.x; i < P; i += blockDim.x) {
                const unsigned j = i ^ stride;
                if (j > i) {
                    const bool up = (i & size) == 0;
                    const bool gt = key[i] > key[j] || (key[i] == key[j] && ord[i] > ord[j]);
                    if (gt == up) {
                        const uint64_t tk = key[i];
                        key[i] = key[j];
                        key[j] = tk;
                        const uint32_t to = ord[i];
                        ord[i] = ord[j];
                        ord[j] = to;
                    }
                }
            }
            __syncthreads();
        }
    }
    // flag bit 7: neighbours i, i+1 are candidates; bit 2: the owner is i+1; bits 0-1: d
    for (unsigned i = threadIdx.x; i + 1 < k; i += blockDim.x) {
        const uint32_t a = ord[i], b = ord[i + 1];
        const uint64_t e = S[a] ^ S[b];
        uint8_t f = 0;
        if (e != 0ull && (e & ~zm) == 0ull) {
            int v1row = -1, q1 = 65;
            for (uint64_t m = e; m; m &= m - 1ull) {
                const int r = __ffsll((long long)m) - 1;
                if (rowq[r] < q1) {
                    q1 = rowq[r];
                    v1row = r;
                }
            }
            const bool a_owns = ((S[a] >> v1row) & 1ull) == 0ull;
            const double2 aj = A[a_owns ? a : b], ar = A[a_owns ? b : a];
            const double nj = sqrt(aj.x * aj.x + aj.y * aj.y);
            if (nj > 0.0) {
                for (int dd = 0; dd < 4; dd++) {
                    const double2 w = ipow_times(aj, dd);
                    const double dx = ar.x - w.x, dy = ar.y - w.y;
                    if (sqrt(dx * dx + dy * dy) <= tol * nj) {
                        f = (uint8_t)(0x80 | (a_owns ? 0 : 4) | dd);
                        break;
                    }
                }
            }
        }
        flag[i] = f;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t np = 0, nk = 0;
        unsigned long long i = 0;
        while (i < k) {
            if (i + 1 < k && (flag[i] & 0x80)) {
                const uint32_t a = ord[i], b = ord[i + 1];
                MfPair p;
                p.owner = (flag[i] & 4) ? b : a;
                p.d = flag[i] & 3u;
                p.e = S[a] ^ S[b];
                pairs[np++] = p;
                i += 2;
            } else {
                keep[nk++] = ord[i];
                i += 1;
            }
        }
        counts[0] = np;
        counts[1] = nk;
    }
}

// dst element i = (ssig[idx[i]], scale * samp[idx[i]]); the count of dst_buf
// becomes m.  Source and destination buffers must differ.
__global__ void __launch_bounds__(kCopyThreads) k_mf_gather(SfDev dst, int dst_buf, const uint64_t* ssig,
                                                            const double2* samp, const uint32_t* idx, uint32_t m,
                                                            double scale) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        const uint32_t j = idx[i];
        dst.sig[dst_buf][i] = ssig[j];
        const double2 a = samp[j];
        dst.amp[dst_buf][i] = make_double2(scale * a.x, scale * a.y);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) dst.kcnt[dst_buf] = m;
}

// Append m exported elements (phase vector, canonical amplitude A) to buffer
// dst_buf of a frame with the same stabilizer matrix, from position off: the
// stored amplitude a satisfies A = g * a * i^ip, ip from elem_amp_phi at the
// anchor of sigma in the destination frame.
__global__ void __launch_bounds__(kCopyThreads) k_mf_import(SfDev dst, int dst_buf, uint64_t off,
                                                            const uint64_t* xsig, const double2* xamp, uint32_t m) {
    if (*dst.status) return;
    const int r = dst.meta[0];
    const double2 g = *dst.g;
    const double gn = g.x * g.x + g.y * g.y;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        uint64_t s[1] = {xsig[i]}, b[1];
        elem_anchor<1>(dst, s, r, b);
        const int ip = elem_amp_phi<1>(dst, s, b, r);
        if (ip < 0 || !(gn > 0.0)) {
            set_status(dst.status, SF_ST_INTERNAL, dst_buf, 41u);
            continue;
        }
        const double2 A = xamp[i];
        // A * conj(g) / |g|^2 * i^{-ip}
        const double2 q = make_double2((A.x * g.x + A.y * g.y) / gn, (A.y * g.x - A.x * g.y) / gn);
        dst.sig[dst_buf][off + i] = s[0];
        dst.amp[dst_buf][off + i] = ipow_times(q, (4 - ip) & 3);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) dst.kcnt[dst_buf] = off + m;
}

unsigned copy_blocks(uint64_t m) {
    const uint64_t b = (m + kCopyThreads - 1) / kCopyThreads;
    return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(b, 1024));
}

}  // namespace

namespace {
unsigned pair_pow2(uint64_t k) {
    unsigned P = 2;
    while (P < k) P <<= 1;
    return P;
}
}  // namespace

size_t sf_mf_pair_smem_bytes(uint64_t k) { return (size_t)pair_pow2(k) * (8 + 4 + 1); }

cudaError_t sf_launch_mf_pair(const SfDev& d, int buf, int stage, uint64_t k, double tol, MfPair* pairs,
                              uint32_t* keep, uint32_t* counts, cudaStream_t s) {
    static const bool attr = cudaFuncSetAttribute(k_mf_pair, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  (int)sf_mf_pair_smem_bytes(SF_MF_MAXK)) == cudaSuccess;
    (void)attr;
    k_mf_pair<<<1, kPairThreads, sf_mf_pair_smem_bytes(k), s>>>(d, buf, stage, tol, pair_pow2(k), pairs, keep,
                                                                 counts);
    return cudaGetLastError();
}

cudaError_t sf_launch_mf_gather(const SfDev& dst, int dst_buf, const uint64_t* ssig, const double2* samp,
                                const uint32_t* idx, uint32_t m, double scale, cudaStream_t s) {
    k_mf_gather<<<copy_blocks(m), kCopyThreads, 0, s>>>(dst, dst_buf, ssig, samp, idx, m, scale);
    return cudaGetLastError();
}

cudaError_t sf_launch_mf_import(const SfDev& dst, int dst_buf, uint64_t off, const uint64_t* xsig,
                                const double2* xamp, uint32_t m, cudaStream_t s) {
    k_mf_import<<<copy_blocks(m), kCopyThreads, 0, s>>>(dst, dst_buf, off, xsig, xamp, m);
    return cudaGetLastError();
}
