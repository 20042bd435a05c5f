// Row-streamed multi-right-hand-side hopping kernel (launch option
// smem_links = 4): the neighbour spinors and links of Eq. (1) reach the SM as
// whole lattice rows copied by the Tensor Memory Accelerator into a ring of
// shared-memory slots, instead of per-thread gathers.
//
// A checkerboard row is the Lx/2 sites of one parity that share (y, z, t);
// its sites have consecutive checkerboard indices, so in every packed plane
// the row's n right-hand sides are one contiguous run of (Lx/2)*n elements.
// A block owns one output row at a time (threads = n right-hand sides x Lx/2
// sites) and consumes it in 7 stages, each one input row:
//   stage 0  the row itself (same y, z, t): neighbours +x and -x of every site
//            (the site to the right or left within the row, by row parity)
//   stage 1, 2  rows y+1, y-1 (periodic);  stage 3, 4  rows z+1, z-1
//   stage 5, 6  rows t+1, t-1 (the time-boundary sign applies when the row
//            wraps in t).
// One thread issues each stage as one 1-D bulk copy per spinor plane
// (cp.async.bulk, completion counted in bytes on an mbarrier) several stages
// ahead; the block waits on the stage's barrier and computes the directions
// of the stage for its (site, right-hand side) elements with the neighbour
// read from shared memory and the link read from global memory (the n
// threads of a site share each link request).  The spinor loads in flight
// take no registers, and the +-x neighbours are read once per row instead of
// once per site.
//
// Every wait on a barrier is bounded (HopArgs::spin_limit clock cycles); a
// block that runs out records PLQ_ERR_TIMEOUT in *HopArgs::kstatus, waits
// (bounded) for the copies it issued, and returns.
#pragma once

namespace plq {

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_test_wait(unsigned long long *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Wait for phase `parity` of the barrier to complete, at most `limit` clock
// cycles; false on expiry.  The first test does not block; the loop then
// waits with try_wait, which may suspend the thread for a while, and checks
// the clock between tries.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity, long long limit) {
    const long long t0 = clock64();
    if (mbar_test_wait(bar, parity)) return true;
    for (;;) {
        if (clock64() - t0 >= limit) return false;
        if (mbar_try_wait(bar, parity)) return true;
    }
}
// 1-D bulk copy global -> shared of `bytes` (a multiple of 16, both addresses
// 16-byte aligned), completion signalled on `bar`
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Shared-memory bytes of one row of spinors (n right-hand sides), rounded up
// to 16: one slot of the ring.
template <int P>
__host__ __device__ inline size_t rows_spinor_bytes(int Lxh, int n) {
    const size_t e = (size_t)Lxh * n;
    return ((e * 16 * spinor_planes<P>() + (P == PLQ_F16 ? e * 4 : 0)) + 15) & ~(size_t)15;
}
template <int P, int R>
__host__ __device__ inline size_t rows_slot_bytes(int Lxh, int n) {
    return rows_spinor_bytes<P>(Lxh, n);
}

// The row's runs can be copied with 16-byte bulk copies (FP16 storage: the
// run of 4-byte site norms must be a multiple of 16 bytes).
template <int P, int R>
inline bool rows_copyable(int Lxh, int n) {
    return !(P == PLQ_F16 && ((long long)Lxh * n) % 4 != 0);
}

// Neighbour spinor (element xh, right-hand side r) from a spinor row in shared
// memory; returns the FP16 site norm (1 for FP32 storage).
template <int P>
__device__ __forceinline__ float row_spinor(const unsigned char *row, int Lxh, int n, int xh, int r,
                                            cx<float> phi[12]) {
    const size_t e = (size_t)xh * n + r, pl = (size_t)Lxh * n;
    if constexpr (P == PLQ_F32) {
        const float4 *p = reinterpret_cast<const float4 *>(row) + e;
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            const float4 v = p[q * pl];
            phi[2 * q] = {v.x, v.y};
            phi[2 * q + 1] = {v.z, v.w};
        }
        return 1.f;
    } else {
        const uint4 *p = reinterpret_cast<const uint4 *>(row) + e;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const uint4 v = p[q * pl];
            const float2 x0 = h2f(v.x), x1 = h2f(v.y), x2 = h2f(v.z), x3 = h2f(v.w);
            phi[4 * q] = {x0.x, x0.y};
            phi[4 * q + 1] = {x1.x, x1.y};
            phi[4 * q + 2] = {x2.x, x2.y};
            phi[4 * q + 3] = {x3.x, x3.y};
        }
        return reinterpret_cast<const float *>(row + 3 * pl * 16)[e];
    }
}

// One direction: project the neighbour with (1 + S gamma_MU), scale (FP16 norm,
// time-boundary sign), multiply by U (BACK = false) or U^dagger, accumulate.
template <int P, int R, int MU, int S, bool BACK>
__device__ __forceinline__ void rows_dir(const unsigned char *sp, const void *lblk, int Vh, int li, int Lxh, int n,
                                         int xn, int r, float sign, cx<float> acc[12]) {
    cx<float> phi[12], h[6], uh[6], u[3][3];
    Link<P, R>::load(lblk, Vh, li, u);  // from global memory; the n threads of a site share the request
    const float sc = row_spinor<P>(sp, Lxh, n, xn, r, phi) * sign;
    project<MU, S>(phi, h);
    if (P == PLQ_F16 || sign != 1.f) {
#pragma unroll
        for (int k = 0; k < 6; ++k) h[k] = {sc * h[k].re, sc * h[k].im};
    }
    if constexpr (BACK) su3_dag_mul(u, h, uh);
    else su3_mul(u, h, uh);
    reconstruct<MU, S>(acc, uh);
}

constexpr int kRowSlots = 8;  // most shared-memory slots of the ring

constexpr int kRowThreads = 512;  // most threads per block (n x Lx/2); 128 registers each

template <int P, int R, int EPI, bool DAG>
__global__ void __launch_bounds__(kRowThreads, 1) hop_rows_kernel(const HopArgs a, int nslot) {
    using T = RealOf<P>;
    extern __shared__ __align__(128) unsigned char rows_smem[];
    __shared__ unsigned long long bars[kRowSlots];
    const Lattice &L = a.lat;
    const int n = a.nrhs, Lxh = L.L[1] >> 1;
    const int r = threadIdx.x, xh = threadIdx.y;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nrows = L.Vh / Lxh;
    const size_t stride = (size_t)L.Vh * n;  // elements of one spinor plane
    const size_t slot_bytes = rows_spinor_bytes<P>(Lxh, n);
    const int par = a.out_parity;
    const char *gbase = static_cast<const char *>(a.gauge);
    const unsigned char *in = static_cast<const unsigned char *>(a.in);
    // stages of this block: 7 per row, rows blockIdx.x, blockIdx.x + gridDim.x, ...
    const int my_rows = blockIdx.x < nrows ? (nrows - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const long long G = 7LL * my_rows;

    // input row and link rows of stage g
    auto stage_rows = [&](long long g, int *ri, int *la_blk, int *la_row, int *lb_blk, int *lb_row, int *ro_out,
                          int *tcoord) {
        const int s = (int)(g % 7);
        const int ro = blockIdx.x + (int)(g / 7) * gridDim.x;
        unsigned y, z;
        const unsigned q = fd_divmod((unsigned)ro, L.div_y, &y);
        const int t = (int)fd_divmod(q, L.div_z, &z);
        const int Ly = L.L[2], Lz = L.L[3], T = L.L[0];
        const int mu = s == 0 ? 1 : s <= 2 ? 2 : s <= 4 ? 3 : 0;
        int nr = ro;
        if (s == 1) nr = ro - (int)y + ((int)y + 1 == Ly ? 0 : (int)y + 1);
        else if (s == 2) nr = ro - (int)y + ((int)y == 0 ? Ly - 1 : (int)y - 1);
        else if (s == 3) nr = ro + (((int)z + 1 == Lz ? 0 : (int)z + 1) - (int)z) * Ly;
        else if (s == 4) nr = ro + (((int)z == 0 ? Lz - 1 : (int)z - 1) - (int)z) * Ly;
        else if (s == 5) nr = ro + ((t + 1 == T ? 0 : t + 1) - t) * Ly * Lz;
        else if (s == 6) nr = ro + ((t == 0 ? T - 1 : t - 1) - t) * Ly * Lz;
        *ri = PLQ_GUARD(a.kstatus, nr, nrows);
        *ro_out = ro;
        *tcoord = t;
        const bool fwd = s == 0 || (s & 1);  // stages 0, 1, 3, 5 need U_mu(x) at the output row
        *la_blk = (fwd ? par : 1 - par) * 4 + mu;
        *la_row = fwd ? ro : nr;
        *lb_blk = (1 - par) * 4 + 1;  // stage 0 only: U_x at the input row
        *lb_row = ro;
    };

    auto issue = [&](long long g) {
        int ri, la_blk, la_row, lb_blk, lb_row, ro, t;
        stage_rows(g, &ri, &la_blk, &la_row, &lb_blk, &lb_row, &ro, &t);
        const int slot = (int)(g % nslot);
        unsigned char *base = rows_smem + (size_t)slot * slot_bytes;
        const int s = (int)(g % 7);
        const size_t e0 = (size_t)ri * Lxh * n, ne = (size_t)Lxh * n;
        constexpr int NP = spinor_planes<P>();
        const unsigned bytes = (unsigned)(ne * 16 * NP + (P == PLQ_F16 ? ne * 4 : 0));
        (void)s;
        mbar_arrive_expect_tx(&bars[slot], bytes);
#pragma unroll
        for (int q = 0; q < NP; ++q)
            bulk_g2s(base + (size_t)q * ne * 16, in + ((size_t)q * stride + e0) * 16, (unsigned)(ne * 16), &bars[slot]);
        if constexpr (P == PLQ_F16)
            bulk_g2s(base + (size_t)NP * ne * 16, in + (size_t)NP * stride * 16 + e0 * 4, (unsigned)(ne * 4),
                     &bars[slot]);
    };

    if (tid == 0) {
        for (int k = 0; k < nslot; ++k) mbar_init(&bars[k], 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    }
    __syncthreads();
    if (tid == 0)
        for (long long g = 0; g < G && g < nslot; ++g) issue(g);

    constexpr int NV = EPI == EPI_XPAY_NORM ? 1 : 0;
    RedAcc<1, 1> racc;
    red_init(racc);
    cx<float> acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = {0.f, 0.f};
    constexpr int SF = DAG ? +1 : -1, SB = -SF;
    long long g = 0;
    bool failed = false;
    for (; g < G; ++g) {
        const int slot = (int)(g % nslot);
        const bool ok = mbar_wait(&bars[slot], (unsigned)((g / nslot) & 1), a.spin_limit);
        if (__syncthreads_or(!ok)) {  // also: every thread is done with stage g - 1
            failed = true;
            break;
        }
        if (tid == 0 && g >= 1 && g - 1 + nslot < G) {
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            issue(g - 1 + nslot);
        }
        const unsigned char *base = rows_smem + (size_t)slot * slot_bytes;
        const int s = (int)(g % 7);
        int ri, la_blk, la_row, lb_blk, lb_row, ro, t;
        stage_rows(g, &ri, &la_blk, &la_row, &lb_blk, &lb_row, &ro, &t);
        unsigned yy, zz;
        fd_divmod(fd_divmod((unsigned)ro, L.div_y, &yy), L.div_z, &zz);
        const int o = (par + (int)yy + (int)zz + t) & 1;  // x = 2 xh + o on the output row
        if (r < n && xh < Lxh) {
            (void)PLQ_GUARD(a.kstatus, ro, nrows);
            const void *la = gbase + (size_t)la_blk * a.gblock;
            const int lrow = la_row * Lxh;
            switch (s) {
            case 0: {
                const int xp = PLQ_GUARD(a.kstatus, o == 0 ? xh : (xh + 1 == Lxh ? 0 : xh + 1), Lxh);
                const int xm = PLQ_GUARD(a.kstatus, o == 1 ? xh : (xh == 0 ? Lxh - 1 : xh - 1), Lxh);
                const void *lb = gbase + (size_t)lb_blk * a.gblock;
                rows_dir<P, R, 1, SF, false>(base, la, L.Vh, lrow + xh, Lxh, n, xp, r, 1.f, acc);
                rows_dir<P, R, 1, SB, true>(base, lb, L.Vh, lb_row * Lxh + xm, Lxh, n, xm, r, 1.f, acc);
                break;
            }
            case 1: rows_dir<P, R, 2, SF, false>(base, la, L.Vh, lrow + xh, Lxh, n, xh, r, 1.f, acc); break;
            case 2: rows_dir<P, R, 2, SB, true>(base, la, L.Vh, lrow + xh, Lxh, n, xh, r, 1.f, acc); break;
            case 3: rows_dir<P, R, 3, SF, false>(base, la, L.Vh, lrow + xh, Lxh, n, xh, r, 1.f, acc); break;
            case 4: rows_dir<P, R, 3, SB, true>(base, la, L.Vh, lrow + xh, Lxh, n, xh, r, 1.f, acc); break;
            case 5: {
                const float sg = (t == L.L[0] - 1 && L.t_bc < 0) ? -1.f : 1.f;
                rows_dir<P, R, 0, SF, false>(base, la, L.Vh, lrow + xh, Lxh, n, xh, r, sg, acc);
                break;
            }
            default: {
                const float sg = (t == 0 && L.t_bc < 0) ? -1.f : 1.f;
                rows_dir<P, R, 0, SB, true>(base, la, L.Vh, lrow + xh, Lxh, n, xh, r, sg, acc);
                break;
            }
            }
            if (s == 6) {
                // the output element (site ro * Lx/2 + xh, right-hand side r)
                const bool frozen = a.st != nullptr && a.st[r].stop;
                if (!frozen) {
                    const long long idx = PLQ_GUARD(a.kstatus, ((long long)ro * Lxh + xh) * n + r, (long long)stride);
                    if (a.nu_h != 0.0 || a.scale_h != 1.0) twist12(acc, (T)a.nu_h, (T)a.scale_h);
                    if constexpr (EPI != EPI_PLAIN) {
                        cx<T> xv[12];
                        Spinor<P>::load(a.x, stride, (size_t)idx, xv);
                        if (a.nu_x != 0.0) twist12(xv, (T)a.nu_x, T(1));
                        const T sa = (T)a.a;
#pragma unroll
                        for (int e = 0; e < 12; ++e) {
                            acc[e].re = fma(sa, acc[e].re, xv[e].re);
                            acc[e].im = fma(sa, acc[e].im, xv[e].im);
                        }
                        if constexpr (NV > 0) {
                            T s0 = 0;
#pragma unroll
                            for (int e = 0; e < 12; ++e) s0 += acc[e].re * acc[e].re + acc[e].im * acc[e].im;
                            racc.add(0, 0, s0);
                        }
                    }
                    Spinor<P>::store(a.out, stride, (size_t)idx, acc);
                }
#pragma unroll
                for (int k = 0; k < 12; ++k) acc[k] = {0.f, 0.f};
            }
        }
    }
    if (failed && tid == 0) {
        atomicCAS(a.kstatus, 0, (int)PLQ_ERR_TIMEOUT);
        // wait (bounded) for the copies this block still has in flight: the
        // stages issued (up to g - 1 + nslot, or nslot - 1 before the first
        // refill) and not yet consumed (from g)
        const long long last = g >= 1 ? g - 1 + nslot : nslot;
        const long long issued = last < G ? last : G;
        for (long long h = g; h < issued; ++h) mbar_wait(&bars[h % nslot], (unsigned)((h / nslot) & 1), 1LL << 31);
    }
    // a block that gave up still takes part in the grid reduction, so the
    // ticket counter completes and is reset for the next launch
    if constexpr (NV > 0) grid_reduce(a.red, racc, blockDim.x);
}

template <int P, int R, int EPI, bool DAG>
plq_status launch_rows_t(const HopArgs &a, cudaStream_t s) {
    const int n = a.nrhs, Lxh = a.lat.L[1] >> 1;
    const int threads = n * Lxh;
    if (threads > kRowThreads || !rows_copyable<P, R>(Lxh, n) || !a.kstatus)
        return set_error(PLQ_ERR_ARG, "the row-streamed kernel does not fit this lattice and nrhs");
    const size_t slot = rows_slot_bytes<P, R>(Lxh, n);
    int dev = 0, sms = 0, smem_max = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const size_t avail = (size_t)smem_max - 2048;  // room for the static shared memory of the kernel
    int nslot = (int)(avail / slot);
    if (a.spt > 0) nslot = a.spt < nslot ? a.spt : nslot;  // sites_per_thread selects the slot count
    if (nslot > kRowSlots) nslot = kRowSlots;
    if (nslot < 2) return set_error(PLQ_ERR_ARG, "the row-streamed kernel's slots do not fit in shared memory");
    const size_t smem = (size_t)nslot * slot;
    auto kern = hop_rows_kernel<P, R, EPI, DAG>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_error(e, "cudaFuncSetAttribute(hop_rows_kernel)");
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    if (e != cudaSuccess) return cuda_error(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor(hop_rows)");
    if (per_sm < 1) return set_error(PLQ_ERR_ARG, "the row-streamed kernel does not fit an SM");
    const long long nrows = a.lat.Vh / Lxh;
    long long grid = (long long)per_sm * sms;
    if (grid > nrows) grid = nrows;
    if (EPI >= EPI_XPAY_NORM && grid > kMaxReduceBlocks) grid = kMaxReduceBlocks;
    kern<<<(int)grid, dim3(n, Lxh), smem, s>>>(a, nslot);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "hop_rows_kernel launch");
    return PLQ_OK;
}

template <int P, int R>
plq_status dispatch_rows(const HopArgs &a, int epi, cudaStream_t s) {
    switch (epi) {
    case EPI_PLAIN:
        return a.dagger ? launch_rows_t<P, R, EPI_PLAIN, true>(a, s) : launch_rows_t<P, R, EPI_PLAIN, false>(a, s);
    case EPI_XPAY:
        return a.dagger ? launch_rows_t<P, R, EPI_XPAY, true>(a, s) : launch_rows_t<P, R, EPI_XPAY, false>(a, s);
    default:
        return a.dagger ? launch_rows_t<P, R, EPI_XPAY_NORM, true>(a, s)
                        : launch_rows_t<P, R, EPI_XPAY_NORM, false>(a, s);
    }
}

}  // namespace plq
