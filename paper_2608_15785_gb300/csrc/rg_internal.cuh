// rg_internal.cuh -- device-side types and helpers shared by the renderer's kernels.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace rg {

constexpr int TILE = 16;                       // default tile edge in pixels (16 x 16 tiles)
constexpr float LN255F = 5.541263545158426f;   // ln 255: alpha = 1/255 in log space, Eq. (23)
// Programmatic dependent launch. The frame's kernels are launched with launch_dependent(): the
// next kernel on the stream may be scheduled while the previous one drains (about 2.7 us less
// per kernel boundary than plain stream order on GB300), and each of these kernels first waits in
// grid_dependency_wait() until the previous grid has completed and its writes are visible, so
// nothing it reads or writes can race with that grid. Without a predecessor launched this way the
// wait returns at once.
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline void launch_dependent(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                             Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, args...); // a failed launch is seen by the caller's cudaGetLastError
}

constexpr unsigned SPIN_LIMIT = 1u << 20;      // bounded device waits: ~1 s of polls with a short sleep

// Error bits of Counters::error / Sticky::error
constexpr unsigned ERR_FE_LOOKBACK = 1u;
constexpr unsigned ERR_SORT_LOOKBACK = 2u;
constexpr unsigned ERR_SCAN_LOOKBACK = 4u;

// Camera as the kernels see it (kernel parameter, uniform across threads).
struct CamDev {
    float R[9];
    float t[3];
    float fx, fy, cx, cy;
    int W, H;
    float zn, zf;
    float bg[3];
    float campos[3];  // camera centre -R^T t (for the SH view direction)
    float limx, limy; // 1.3 * tan(half field of view), FP32 pinned: 1.3f * ((0.5f * W) / fx)
    int tw, th;       // tile shape in pixels: 16 x 16, 32 x 8 or 8 x 32 (tw * th = 256)
    int tw_log2;      // log2(tw): thread t of a tile block owns column t & (tw - 1)
    int th_log2;      // log2(th); pixel x >= 0 lies in tile column x >> tw_log2 (= x / tw)
};

// Tile grid and resolution-adaptive key split (Sec. IV-A.2).
struct Layout {
    int tiles_x, tiles_y;
    int b_t, b_d;
    unsigned qmax;       // 2^b_d - 1
    float depth_scale;   // fl32((2^b_d - 1) / (zf - zn)) computed in FP64
};

// Per-frame device counters (zeroed at the start of every frame).
struct Counters {
    unsigned long long n_entries_total; // entries the front end wanted to emit
    unsigned n_entries;                 // entries present in the key arrays (<= capacity)
    unsigned n_visible;
    unsigned overflow;
    unsigned error;
    unsigned fe_block_ctr;   // virtual block ids of the fused front end / exact scan
    unsigned sort_tile_ctr[8];
    unsigned n_front;
    unsigned pad;
    unsigned long long n_pairs;  // rasterizer work counters (counting launches only)
    unsigned long long n_blends;
};

// Sticky flags across frames (cleared by rg_scene_check).
struct Sticky {
    unsigned overflow;
    unsigned error;
};

// Status word of the decoupled look-back (64-bit: 2 flag bits + 62-bit value).
constexpr unsigned long long LB_AGG = 1ull << 62;
constexpr unsigned long long LB_PRE = 2ull << 62;
constexpr unsigned long long LB_VAL = (1ull << 62) - 1ull;

__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long* p)
{
    return *reinterpret_cast<const volatile unsigned long long*>(p);
}
__device__ __forceinline__ void st_volatile_u64(unsigned long long* p, unsigned long long v)
{
    *reinterpret_cast<volatile unsigned long long*>(p) = v;
}

// Single-pass decoupled look-back (warp-parallel). Called by all 32 lanes of ONE
// warp of the block; returns the exclusive prefix of `aggregate` over all lower
// virtual block ids in every lane. Waits are bounded: on time-out the error bit
// is raised (sticky too) and the missing predecessors count as zero.
__device__ __forceinline__ unsigned long long lookback_exclusive(unsigned long long* status, unsigned vb,
                                                                 unsigned long long aggregate, Counters* ctr,
                                                                 Sticky* sticky, unsigned errbit)
{
    const unsigned lane = threadIdx.x & 31u;
    if (vb == 0) {
        if (lane == 0) st_volatile_u64(&status[0], LB_PRE | aggregate);
        return 0ull;
    }
    if (lane == 0) st_volatile_u64(&status[vb], LB_AGG | aggregate);
    unsigned long long excl = 0ull;
    long long top = (long long)vb - 1;
    bool timed_out = false;
    while (true) {
        long long idx = top - (long long)lane;
        unsigned long long s = LB_PRE; // before block 0: prefix 0
        if (idx >= 0) {
            unsigned spins = 0;
            s = ld_volatile_u64(&status[idx]);
            while ((s >> 62) == 0ull) {
                if (++spins > SPIN_LIMIT) {
                    timed_out = true;
                    s = LB_PRE;
                    break;
                }
                __nanosleep(64);
                s = ld_volatile_u64(&status[idx]);
            }
        }
        const unsigned pmask = __ballot_sync(0xffffffffu, (s >> 62) == 2ull);
        const int stop = pmask ? (__ffs(pmask) - 1) : 32;
        unsigned long long v = ((int)lane <= stop) ? (s & LB_VAL) : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        excl += v;
        if (pmask) break;
        top -= 32;
    }
    if (__any_sync(0xffffffffu, timed_out) && lane == 0) {
        atomicOr(&ctr->error, errbit);
        atomicOr(&sticky->error, errbit);
    }
    if (lane == 0) st_volatile_u64(&status[vb], LB_PRE | (excl + aggregate));
    return excl;
}

// ---------------------------------------------------------------------------
// FP32 pinned-order projection and binning (every step one IEEE operation;
// the CPU oracle evaluates the same sequence, so culling, tile rectangles and
// keys are bit-exact).
// ---------------------------------------------------------------------------
struct Binned {
    float z, u, v;
    float sa, sb, sc;   // Sigma' = [[sa, sb], [sb, sc]] including the 0.3 dilation
    float det;          // det Sigma' by the Lagrange identity (pinned)
    float tt;           // RoofGS: ellipse level t = 2 (log o + ln 255)
    float xl, xh, yl, yh; // pixel-centre box, clipped to the image
    int tx0, ty0, tx1, ty1;
};

#define FM(a, b) __fmul_rn((a), (b))
#define FA(a, b) __fadd_rn((a), (b))
#define FS(a, b) __fsub_rn((a), (b))
#define FD(a, b) __fdiv_rn((a), (b))

__device__ __forceinline__ float view_z(const CamDev& c, float mx, float my, float mz)
{
    return FA(FA(FA(FM(c.R[6], mx), FM(c.R[7], my)), FM(c.R[8], mz)), c.t[2]);
}

// Projection, EWA covariance, box and tile rectangle. snug = RoofGS box (exact
// alpha = 1/255 ellipse, needs log o) else the 3-sigma box of plain 3DGS.
// Returns false if culled or if the rectangle is empty. pz has been computed
// by view_z and passed the depth-interval test.
__device__ __forceinline__ bool project_bin(const CamDev& c, float mx, float my, float mz, float pz, float qw,
                                            float qx, float qy, float qz, float s0, float s1, float s2, bool snug,
                                            float logo, Binned& b)
{
    const float px = FA(FA(FA(FM(c.R[0], mx), FM(c.R[1], my)), FM(c.R[2], mz)), c.t[0]);
    const float py = FA(FA(FA(FM(c.R[3], mx), FM(c.R[4], my)), FM(c.R[5], mz)), c.t[1]);
    b.z = pz;
    const float n2 = FA(FA(FA(FM(qw, qw), FM(qx, qx)), FM(qy, qy)), FM(qz, qz));
    if (!(n2 > 0.0f)) return false;
    const float rn = __fsqrt_rn(n2);
    const float w = FD(qw, rn), x = FD(qx, rn), y = FD(qy, rn), z = FD(qz, rn);
    const float xx = FM(x, x), yy = FM(y, y), zz = FM(z, z);
    const float xy = FM(x, y), xz = FM(x, z), yz = FM(y, z);
    const float wx = FM(w, x), wy = FM(w, y), wz = FM(w, z);
    float Q[9];
    Q[0] = FS(1.0f, FM(2.0f, FA(yy, zz)));
    Q[1] = FM(2.0f, FS(xy, wz));
    Q[2] = FM(2.0f, FA(xz, wy));
    Q[3] = FM(2.0f, FA(xy, wz));
    Q[4] = FS(1.0f, FM(2.0f, FA(xx, zz)));
    Q[5] = FM(2.0f, FS(yz, wx));
    Q[6] = FM(2.0f, FS(xz, wy));
    Q[7] = FM(2.0f, FA(yz, wx));
    Q[8] = FS(1.0f, FM(2.0f, FA(xx, yy)));
    const float s[3] = {s0, s1, s2};
    float M[9];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int k = 0; k < 3; k++) M[3 * i + k] = FM(Q[3 * i + k], s[k]);

    const float xzr = FD(px, pz), yzr = FD(py, pz);
    const float cxz = fminf(c.limx, fmaxf(-c.limx, xzr));
    const float cyz = fminf(c.limy, fmaxf(-c.limy, yzr));
    const float j00 = FD(c.fx, pz), j11 = FD(c.fy, pz);
    const float j02 = -FM(j00, cxz), j12 = -FM(j11, cyz);
    float A[6];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        A[k] = FA(FM(j00, c.R[k]), FM(j02, c.R[6 + k]));
        A[3 + k] = FA(FM(j11, c.R[3 + k]), FM(j12, c.R[6 + k]));
    }
    float U[6];
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int k = 0; k < 3; k++)
            U[3 * i + k] = FA(FA(FM(A[3 * i], M[k]), FM(A[3 * i + 1], M[3 + k])), FM(A[3 * i + 2], M[6 + k]));
    const float n0 = FA(FA(FM(U[0], U[0]), FM(U[1], U[1])), FM(U[2], U[2]));
    const float n1 = FA(FA(FM(U[3], U[3]), FM(U[4], U[4])), FM(U[5], U[5]));
    const float sa = FA(n0, 0.3f);
    const float sc = FA(n1, 0.3f);
    const float sb = FA(FA(FM(U[0], U[3]), FM(U[1], U[4])), FM(U[2], U[5]));
    const float u = FA(FM(c.fx, xzr), c.cx);
    const float v = FA(FM(c.fy, yzr), c.cy);
    float rx, ry;
    if (!snug) {
        const float h = FM(0.5f, FS(sa, sc));
        const float disc = __fsqrt_rn(FA(FM(h, h), FM(sb, sb)));
        const float lmax = FA(FM(0.5f, FA(sa, sc)), disc);
        rx = ry = ceilf(FM(3.0f, __fsqrt_rn(lmax)));
    } else {
        const float tt = FM(2.0f, FA(logo, LN255F));
        rx = __fsqrt_rn(FM(tt, sa));
        ry = __fsqrt_rn(FM(tt, sc));
    }
    b.u = u;
    b.v = v;
    b.sa = sa;
    b.sb = sb;
    b.sc = sc;
    if (!isfinite(u) || !isfinite(v) || !isfinite(rx) || !isfinite(ry)) return false;
    const float xl = fmaxf(ceilf(FS(u, rx)), 0.0f);
    const float xh = fminf(floorf(FA(u, rx)), (float)(c.W - 1));
    const float yl = fmaxf(ceilf(FS(v, ry)), 0.0f);
    const float yh = fminf(floorf(FA(v, ry)), (float)(c.H - 1));
    if (xl > xh || yl > yh) return false;
    b.xl = xl;
    b.xh = xh;
    b.yl = yl;
    b.yh = yh;
    b.tx0 = (int)xl >> c.tw_log2; // xl, xh, yl, yh >= 0: the shifts are the divisions by tw, th
    b.tx1 = (int)xh >> c.tw_log2;
    b.ty0 = (int)yl >> c.th_log2;
    b.ty1 = (int)yh >> c.th_log2;
    // det Sigma' = |U0 x U1|^2 + 0.3 (|U0|^2 + |U1|^2) + 0.09 (Lagrange identity:
    // no cancellation for thin Gaussians)
    const float c0 = FS(FM(U[1], U[5]), FM(U[2], U[4]));
    const float c1 = FS(FM(U[2], U[3]), FM(U[0], U[5]));
    const float c2 = FS(FM(U[0], U[4]), FM(U[1], U[3]));
    b.det = FA(FA(FA(FA(FM(c0, c0), FM(c1, c1)), FM(c2, c2)), FM(0.3f, FA(n0, n1))), 0.09f);
    b.tt = snug ? FM(2.0f, FA(logo, LN255F)) : 0.0f;
    return true;
}

// Per-Gaussian constants of the RoofGS per-row tile test: for a band of rows the
// x-extent of the ellipse {d : d^T Sigma'^-1 d <= t} is u + c dy +- k sqrt(t - dy^2 / Sigma'_yy)
// with c = Sigma'_xy / Sigma'_yy, k = sqrt(det / Sigma'_yy); its right-most point is at
// dy = Sigma'_xy sqrt(t / Sigma'_xx) (left-most at minus that).
struct RowTest {
    float u, v, tt, isc, ys, cc, kk, xl, xh, yl, yh;
    int ty0, ty1;
};

__device__ __forceinline__ RowTest row_test(const Binned& b)
{
    RowTest r;
    r.u = b.u;
    r.v = b.v;
    r.tt = b.tt;
    r.isc = FD(1.0f, b.sc);
    r.ys = FM(b.sb, __fsqrt_rn(FD(b.tt, b.sa)));
    r.cc = FD(b.sb, b.sc);
    r.kk = __fsqrt_rn(FD(b.det, b.sc));
    r.xl = b.xl;
    r.xh = b.xh;
    r.yl = b.yl;
    r.yh = b.yh;
    r.ty0 = b.ty0;
    r.ty1 = b.ty1;
    return r;
}

// The per-row test as the other lanes of a warp read it (shared memory): the
// constants and the first tile row.
struct RowTestS {
    float u, v, tt, isc, ys, cc, kk, xl, xh, yl, yh;
    int ty0;
};

__device__ __forceinline__ RowTestS shared_row_test(const RowTest& r)
{
    return RowTestS{r.u, r.v, r.tt, r.isc, r.ys, r.cc, r.kk, r.xl, r.xh, r.yl, r.yh, r.ty0};
}

// Tile range [txa, txb] of tile row ty: the ellipse's x-extent over the row's band of
// pixel centres, clipped to the box (reading of the Speedy-Splat culling, Sec. IV-A.3).
// Returns false if no pixel centre of the band lies in it. Pinned FP32 order.
template <class G>
__device__ __forceinline__ bool row_range(const G& g, int ty, int tw_log2, int th, int& txa, int& txb)
{
    const float ya = fmaxf((float)(ty * th), g.yl);
    const float yb = fminf((float)(ty * th + th - 1), g.yh);
    const float d0 = FS(ya, g.v), d1 = FS(yb, g.v);
    const float dmax = fminf(fmaxf(g.ys, d0), d1);
    const float dmin = fminf(fmaxf(-g.ys, d0), d1);
    const float wr = __fsqrt_rn(fmaxf(FS(g.tt, FM(FM(dmax, dmax), g.isc)), 0.0f));
    const float wl = __fsqrt_rn(fmaxf(FS(g.tt, FM(FM(dmin, dmin), g.isc)), 0.0f));
    const float xr = FA(FA(g.u, FM(g.cc, dmax)), FM(g.kk, wr));
    const float xf = FS(FA(g.u, FM(g.cc, dmin)), FM(g.kk, wl));
    const float a0 = fmaxf(ceilf(xf), g.xl);
    const float a1 = fminf(floorf(xr), g.xh);
    if (!(a0 <= a1)) return false;
    txa = (int)a0 >> tw_log2; // 0 <= a0 <= a1: the division by the tile width
    txb = (int)a1 >> tw_log2;
    return true;
}

// Quantized depth of Eq. (9): clamp(floor((d - zn) * (2^b_d - 1) / (zf - zn)), 0, 2^b_d - 1)
__device__ __forceinline__ unsigned quantize_depth(float pz, float zn, const Layout& L)
{
    float dq = FM(FS(pz, zn), L.depth_scale);
    dq = fmaxf(dq, 0.0f);
    const float fq = floorf(dq);
    return (fq >= (float)L.qmax) ? L.qmax : (unsigned)fq;
}

// ---------------------------------------------------------------------------
// Real spherical harmonics, degree <= 3, index k = l^2 + l + m, no
// Condon-Shortley phase (Y_{1,-1}, Y_{1,0}, Y_{1,1} are positive multiples of
// y, z, x).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void sh_basis(float x, float y, float z, float Y[16])
{
    Y[0] = 0.28209479177387814f;
    Y[1] = 0.4886025119029199f * y;
    Y[2] = 0.4886025119029199f * z;
    Y[3] = 0.4886025119029199f * x;
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = 1.0925484305920792f * x * y;
    Y[5] = 1.0925484305920792f * y * z;
    Y[6] = 0.31539156525252005f * (3.0f * zz - 1.0f);
    Y[7] = 1.0925484305920792f * x * z;
    Y[8] = 0.5462742152960396f * (xx - yy);
    Y[9] = 0.5900435899266435f * y * (3.0f * xx - yy);
    Y[10] = 2.890611442640554f * x * y * z;
    Y[11] = 0.4570457994644658f * y * (5.0f * zz - 1.0f);
    Y[12] = 0.3731763325901154f * z * (5.0f * zz - 3.0f);
    Y[13] = 0.4570457994644658f * x * (5.0f * zz - 1.0f);
    Y[14] = 1.445305721320277f * z * (xx - yy);
    Y[15] = 0.5900435899266435f * x * (xx - 3.0f * yy);
}

__device__ __forceinline__ void view_dir(const CamDev& c, float mx, float my, float mz, float& dx, float& dy,
                                         float& dz)
{
    dx = mx - c.campos[0];
    dy = my - c.campos[1];
    dz = mz - c.campos[2];
    const float inv = rsqrtf(dx * dx + dy * dy + dz * dz);
    dx *= inv;
    dy *= inv;
    dz *= inv;
}

__device__ __forceinline__ float clamp01(float x) { return fminf(fmaxf(x, 0.0f), 1.0f); }

// ---------------------------------------------------------------------------
// Double-float arithmetic: a value carried as the unevaluated sum hi + lo of two
// FP32 numbers (Dekker 1971: the exact product by a fused multiply-add; Knuth's
// two-sum; the compensated dot product of Ogita, Rump and Oishi 2005, which is
// as accurate as evaluation in twice the working precision). Exact mode carries
// the projected mean this way: in FP32 alone u has an error of ~1e-3 pixel at
// 4K (the camera transform and the division), which moves the exponent of a
// small Gaussian by up to 1e-2.
// ---------------------------------------------------------------------------
struct DF {
    float hi, lo;
};

__device__ __forceinline__ DF two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ DF fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ DF two_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

// r0 m0 + r1 m1 + r2 m2 + t
__device__ __forceinline__ DF dot3_df(float r0, float r1, float r2, float m0, float m1, float m2, float t)
{
    const DF p0 = two_prod(r0, m0), p1 = two_prod(r1, m1), p2 = two_prod(r2, m2);
    const DF s1 = two_sum(p0.hi, p1.hi);
    const DF s2 = two_sum(s1.hi, p2.hi);
    const DF s3 = two_sum(s2.hi, t);
    const float lo = __fadd_rn(__fadd_rn(__fadd_rn(p0.lo, p1.lo), __fadd_rn(p2.lo, s1.lo)), __fadd_rn(s2.lo, s3.lo));
    return two_sum(s3.hi, lo);
}

// (a.hi + a.lo) / (b.hi + b.lo): quotient q1 = a.hi / b.hi, remainder a - q1 b
// (a.hi - hi(q1 b.hi) is exact), correction q2 = remainder / b.hi
__device__ __forceinline__ DF div_df(DF a, DF b)
{
    const float q1 = __fdiv_rn(a.hi, b.hi);
    const DF p = two_prod(q1, b.hi);
    float r = __fsub_rn(a.hi, p.hi);
    r = __fsub_rn(r, p.lo);
    r = __fadd_rn(r, a.lo);
    r = __fmaf_rn(-q1, b.lo, r);
    return fast_two_sum(q1, __fdiv_rn(r, b.hi));
}

// f q + c
__device__ __forceinline__ DF affine_df(float f, DF q, float c)
{
    const DF p = two_prod(f, q.hi);
    const float plo = __fmaf_rn(f, q.lo, p.lo);
    const DF s = two_sum(p.hi, c);
    return two_sum(s.hi, __fadd_rn(s.lo, plo));
}

// Projected mean u = fx x/z + cx, v = fy y/z + cy of (x, y, z) = R m + t as
// double-floats: (u.hi, u.lo, v.hi, v.lo).
__device__ __forceinline__ float4 project_mean_df(const CamDev& c, float mx, float my, float mz)
{
    const DF x = dot3_df(c.R[0], c.R[1], c.R[2], mx, my, mz, c.t[0]);
    const DF y = dot3_df(c.R[3], c.R[4], c.R[5], mx, my, mz, c.t[1]);
    const DF z = dot3_df(c.R[6], c.R[7], c.R[8], mx, my, mz, c.t[2]);
    const DF u = affine_df(c.fx, div_df(x, z), c.cx);
    const DF v = affine_df(c.fy, div_df(y, z), c.cy);
    return make_float4(u.hi, u.lo, v.hi, v.lo);
}

// Exact-mode exponent p = -1/2 d^T Sigma'^-1 d of Eq. (10) at the pixel offset
// d = (dx, dy) from the mean, with the quadratic form completed in dx:
//   d^T Sigma'^-1 d = (Sigma'_yy / det) (dx - c dy)^2 + dy^2 / Sigma'_yy,  c = Sigma'_xy / Sigma'_yy.
// Both terms are non-negative, so a thin Gaussian does not cancel large terms as
// the expanded a dx^2 + b dx dy + c dy^2 does. quad = (-Sigma'_yy / (2 det), c,
// -1/(2 Sigma'_yy), opacity); m = (u.hi - x0, u.lo, v.hi - y0, v.lo) with the
// pixel at (x0 + lx, y0 + ly).
__device__ __forceinline__ float exact_power(const float4& m, const float4& quad, float lx, float ly)
{
    const float dy = __fsub_rn(__fsub_rn(ly, m.z), m.w);
    const float t = __fsub_rn(__fmaf_rn(-quad.y, dy, __fsub_rn(lx, m.x)), m.y);
    return __fmaf_rn(__fmul_rn(quad.x, t), t, __fmul_rn(__fmul_rn(quad.z, dy), dy));
}

// ---------------------------------------------------------------------------
// Host-side launchers (defined in the .cu files).
// ---------------------------------------------------------------------------
// The front end's blocks add their digit counts to one of these copies (block id
// modulo the count): the atomics spread over many L2 lines instead of 512 words.
constexpr int FE_HIST_COPIES = 16;

struct FrontendArgs {
    const unsigned* order; // [N] Gaussian processed by thread slot i (depth order), or null (index order)
    const float4* geoA;    // [N] (mean.xyz, log o)
    const uint4* geoB;     // [N] FP16 (qw,qx | qy,qz | s0,s1 | s2,g)
    const uint4* shq;      // [N][3] INT8 SH codes, 48 contiguous bytes per Gaussian (byte j = 3k + c)
    float band_scale[12];  // s_{d,c}, [d][c]
    int per_gauss_scale;
    int sh_degree;
    long long n;
    CamDev cam;
    Layout lay;
    float4* rec;           // [N][2] raster record
    unsigned* keys;        // [cap] 32-bit keys (tile << b_d | q_d), unless keys16 is set
    unsigned short* keys16; // [cap] or null: the tile id alone (b_t <= 16; the entries come out in
                            // depth order, so the 32-bit key follows from the tile and the value)
    unsigned* vals;        // [cap]
    long long cap;
    unsigned long long* status; // [ceil(N/256)]
    Counters* ctr;
    Sticky* sticky;
    unsigned* hist;             // [FE_HIST_COPIES][2][256] digit counts of the tile field, or null
    int hist_passes;            // 0, 1 or 2: 8-bit digits of the tile id counted (b_t <= 16)
    // Row-bucketed front end (launch_frontend_rows): rows > 0 tile rows (at most 256, as are
    // the tile columns); the entries carry the column-major 16-bit key tx << 8 | ty and come
    // out grouped by tile row, which leaves one 8-bit sort pass (the column) to the sort
    int rows;
    unsigned* row_n;             // [N] tile rows of the Gaussian of each slot (0: none)
    float4* row_rt;              // [3][N] its row test (RowTestS as three float4 planes)
    unsigned* row_cnt;           // [rows][blocks] entries of each tile row per block, then their
                                 // exclusive prefix over the blocks (saturated at 2^31 - 1)
    unsigned long long* row_tot; // [rows] entries of each tile row
};
void launch_frontend_fused(const FrontendArgs& a, cudaStream_t s);
// count kernel -> per-row scan of the block counts -> scatter kernel (a.rows > 0)
void launch_frontend_rows(const FrontendArgs& a, cudaStream_t s);

// Views of a batch rendered by one launch of a stage (the batch's fused path).
constexpr int MAX_BATCH_VIEWS = 32;

struct FrontendViews {
    FrontendArgs views[MAX_BATCH_VIEWS];
    unsigned block_prefix[MAX_BATCH_VIEWS + 1]; // first block of each view; [n_views] = all blocks
    int n_views;
    unsigned* claim;                            // zeroed before the launch
};
// kernel parameters are limited to 32,764 bytes
static_assert(sizeof(FrontendViews) <= 32000, "the views' front-end arguments must fit the kernel parameters");
// one grid over the Gaussians of every view: block_prefix[v] = sum over earlier views of
// ceil(n / frontend_block_threads())
void launch_frontend_views(const FrontendViews& m, cudaStream_t s);
// threads per block of the fused front end (one look-back status word per block)
int frontend_block_threads();
// quantized depth (Eq. (9)) of every Gaussian as a sort key, Gaussian index as value;
// culled Gaussians get 2^b_d - 1 (the fused front end skips them); writes n to ctr and
// adds the keys' 8-bit digit counts of `passes` (<= 4) passes to hist [passes][256]
// look-back status words of a one-sweep pass over n keys of key_bytes bytes (256 per sort tile)
long long sort_status_words(int key_bytes, long long n);
// quantized depth keys and their digit counts; also clears status0[0 .. sort_status_words(4, n))
void launch_depth_keys(const FrontendArgs& a, unsigned* keys, unsigned* vals, Counters* ctr, unsigned* hist,
                       int passes, unsigned* status0, cudaStream_t s);

struct ExactArgs {
    const float* means;
    const float* scales;
    const float* quats;
    const float* opac;
    const float* sh;
    int sh_degree;
    long long n;
    CamDev cam;
    Layout lay;
    float4* mean2;         // [N] projected mean as double-floats (u.hi, u.lo, v.hi, v.lo)
    float* depth;
    float4* quad;          // [N] (-Sigma'_yy / (2 det), Sigma'_xy / Sigma'_yy, -1 / (2 Sigma'_yy), opacity)
    float* rgb;            // [N][3]
    int4* rect;            // [N] tx0, ty0, tx1, ty1
    unsigned* touched;     // [N]
    unsigned* offsets;     // [N] exclusive scan of touched
    unsigned long long* keys; // [cap]
    unsigned* vals;
    long long cap;
    unsigned long long* status; // scan look-back
    Counters* ctr;
    Sticky* sticky;
    unsigned* hist;        // [FE_HIST_COPIES][8][256] the sort's digit counts (passes 0-3: depth bits,
                           // 4-5: tile bits), counted by the duplicate kernel, or null
    int tile_passes;       // 1 or 2 tile-bit passes (b_t <= 16) when hist is set
};
void launch_exact_preprocess(const ExactArgs& a, cudaStream_t s);
void launch_exact_scan(const ExactArgs& a, cudaStream_t s);
void launch_exact_duplicate(const ExactArgs& a, cudaStream_t s);

// How a warp finds the lanes that hold the same digit (the ranking of a one-sweep pass):
// match_any (few distinct digits per warp), or a per-warp bit mask per digit in shared
// memory that every lane ORs its bit into (many distinct digits).
enum { SORT_RANK_MATCH = 0, SORT_RANK_PEERS = 1 };
constexpr unsigned sort_rank_modes(int m0, int m1 = 0, int m2 = 0, int m3 = 0)
{
    return (unsigned)m0 | ((unsigned)m1 << 2) | ((unsigned)m2 << 4) | ((unsigned)m3 << 6);
}

struct SortArgs {
    void* keys[2];        // ping-pong key buffers (uint32 or uint64)
    unsigned* vals[2];
    long long cap;
    int key_bytes;        // 2 (16-bit tile ids), 4 or 8
    int passes;           // 8-bit digits
    int bit0;             // lowest key bit sorted (digit p = bits bit0 + 8p ..)
    unsigned rank_modes;  // 2 bits per pass p (bits 2p, 2p+1): how warps rank the digits of pass p,
                          // SORT_RANK_MATCH or SORT_RANK_PEERS
    unsigned* hist;       // [8][256]
    unsigned* hist_pre;   // [passes][256] digit counts from the producer of the keys, or null
    const unsigned* hist_copies; // [FE_HIST_COPIES][hist_copy_stride][256] the producer's partial counts
                                 // (summed into hist_pre), or null if hist_pre is complete already
    int hist_copy_stride;        // passes per copy of hist_copies
    unsigned* status[2];  // [max_tiles][256] look-back status per pass (alternating)
    long long max_tiles;
    int hist_done;        // 1: hist_pre is complete and status[0] clear when the sort starts (the
                          // producer of the keys did both): no histogram kernel
    Counters* ctr;
    Sticky* sticky;
};
int sort_tile_items();
void launch_sort(const SortArgs& a, cudaStream_t s, cudaEvent_t ev_after_hist);

struct RangeArgs {
    const void* keys;
    int key_bytes;
    int tile_shift;  // key >> tile_shift = tile id
    long long ntiles;
    uint2* ranges;
    Counters* ctr;
};
void launch_ranges(const RangeArgs& a, cudaStream_t s);

struct RasterArgs {
    const uint2* ranges;
    // RoofGS: when set, every tile block finds its own [start, end) in the sorted keys
    // (tile id = key >> tile_shift, n_entries from the counters) and writes it to
    // ranges_out; `ranges` is then unused
    const unsigned* skeys;
    const unsigned short* skeys16; // instead of skeys: 16-bit tile ids (tile_shift 0)
    int key_cols;                  // skeys16 hold the column-major key tx << 8 | ty
    int tile_shift;
    uint2* ranges_out;
    const Counters* ctr;  // frame counters (n_entries) for the search
    const unsigned* vals;
    long long n;          // Gaussians (values are indices below n)
    int tiles_x, tiles_y;
    CamDev cam;
    float* out;           // [3][H][W]
    // RoofGS
    const float4* rec;
    int fast_exp;
    int ppt;              // pixels per thread: 1, 2 (Eq. (20)) or 4
    // exact
    const float4* mean2;
    const float4* quad;
    const float* rgb;
    Counters* count;      // non-null: count evaluated / blended pairs (separate kernel variant)
};
void launch_raster_roofgs(const RasterArgs& a, cudaStream_t s);

struct RasterViews {
    RasterArgs views[MAX_BATCH_VIEWS];          // RoofGS tile-search arguments of each view
    unsigned tile_prefix[MAX_BATCH_VIEWS + 1];  // first item of each view; [n_views] = all tiles
    int n_views;
    unsigned* claim;                            // zeroed before the launch
};
static_assert(sizeof(RasterViews) <= 32000, "the views' rasterizer arguments must fit the kernel parameters");
// one persistent launch over the (view, tile) items of every view
void launch_raster_views(const RasterViews& m, int fast_exp, int ppt, cudaStream_t s);
void launch_raster_exact(const RasterArgs& a, cudaStream_t s);
void launch_fast_exp_eval(const float* P, float* out, long long n, cudaStream_t s);

// Per-tile counting sort of 16-bit-tile-id entries (tilesort.cu): stable, one scatter.
struct TileSortArgs {
    const unsigned short* keys16; // [n] tile ids, entries in (depth code, Gaussian) order
    const unsigned* vals;         // [n]
    unsigned* vout;               // [n] the values grouped by tile, order kept within a tile
    unsigned* M;                  // [chunks][T] per-chunk tile counts, then their column prefix
    unsigned* tot;                // [T] tile totals, then each tile's first slot
    uint2* ranges;                // [T] [first, end) of every tile, [0, 0) if empty
    int T;                        // tiles of the frame
    int chunks;                   // tilesort_chunks(T)
    const Counters* ctr;          // n_entries
};
// tiles the shared-memory offsets allow (one 4-byte offset per tile in a block)
int tilesort_max_tiles();
// chunks (blocks) for T tiles: SMs x the blocks per SM the shared memory allows; 0 if T is too large
int tilesort_chunks(int T);
// bytes of the C x T count matrix, and their maximum over every T
size_t tilesort_matrix_bytes(int T);
size_t tilesort_matrix_bytes_max();
void launch_tile_counting_sort(const TileSortArgs& a, cudaStream_t s);

struct BackwardArgs {
    // forward state of the frame (exact mode)
    const uint2* ranges;
    const unsigned* vals;
    long long n;
    int tiles_x, tiles_y;
    CamDev cam;
    const float4* mean2;
    const float4* quad;
    const float* rgb;
    const unsigned* touched;
    // scene attributes (FP32)
    const float* means;
    const float* scales;
    const float* quats;
    const float* sh;
    int sh_degree;
    // dL/dimage [3][H][W] and per-Gaussian image-space gradients [n][9]:
    // d(u, v), d(conic A, B, C), d(opacity), d(rgb)
    const float* dL_dimg;
    float* gbuf;
    // outputs
    float* dmeans;
    float* dscales;
    float* dquats;
    float* dopac;
    float* dsh;
};
void launch_raster_backward(const BackwardArgs& a, cudaStream_t s);
void launch_preprocess_backward(const BackwardArgs& a, cudaStream_t s);

// SMs of the current device (looked up once per device).
int device_sm_count();

// Sets the message that rg_last_error() returns on this thread.
void set_last_error(const char* msg);

// Scene creation kernels
void launch_check_finite(const float* p, long long count, unsigned* flag, cudaStream_t s);
void launch_sh_absmax(const float* sh, long long n, unsigned* maxbits /*[12]*/, cudaStream_t s);
void launch_compact(const float* means, const float* scales, const float* quats, const float* logo,
                    const float* sh, long long n, const float* band_scale /*host [12]*/, int per_gauss,
                    float4* geoA, uint4* geoB, uint4* shq, cudaStream_t s);

} // namespace rg
