// backward.cu -- gradients of the exact-mode (plain 3DGS) render.
//
// Not part of the paper (which only renders); it differentiates the forward of
// Sec. III-D: C = sum_i c_i alpha_i T_i + T_final bg, alpha_i = min(0.99, o_i exp(p_i))
// (Eqs. (7), (10)-(12)), T_{i+1} = T_i (1 - alpha_i).
//
//  * k_raster_backward: one block per 16x16 tile. Each pixel first replays its
//    front-to-back blend to find its final transmittance and last blended pair
//    (transmittance is recomputed, never stored), then walks the same pairs back to
//    front: T_i = T_{i+1} / (1 - alpha_i), R (colour behind pair i) grows by
//    c_i alpha_i T_i, and
//        dC/dc_i = alpha_i T_i,   dC/dalpha_i = c_i T_i - R_i / (1 - alpha_i).
//    Per-Gaussian sums of d(u, v), d(conic), d(opacity), d(rgb) are reduced over the
//    warp before one atomic add per warp.
//  * k_preprocess_backward: one thread per Gaussian, the chain rule through the
//    conic (inverse of Sigma'), Sigma' = (J W M)(J W M)^T + 0.3 I with M = R(q) diag(s),
//    the perspective Jacobian J (tangent clamp included), the projected mean and the
//    view-dependent SH colour (coefficients and view direction).
#include "rg_internal.cuh"

namespace rg {

constexpr int B_THREADS = 256;

// forward per-pair opacity of the exact rasterizer (the same exponent, exact_power);
// false if the pair is skipped. m is the mean shifted to the tile origin, (lx, ly)
// the pixel in the tile; dx = u - x, dy = v - y are returned for the gradients
__device__ __forceinline__ bool exact_alpha(const float4& m, const float4& q, float lx, float ly, float& dx, float& dy,
                                            float& e, float& alpha)
{
    const float power = exact_power(m, q, lx, ly);
    dx = (m.x - lx) + m.y;
    dy = (m.z - ly) + m.w;
    e = expf(power);
    alpha = fminf(0.99f, q.w * e);
    return alpha >= 1.0f / 255.0f;
}

__device__ __forceinline__ float warp_red(float x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

__global__ void __launch_bounds__(B_THREADS) k_raster_backward(BackwardArgs a)
{
    __shared__ unsigned s_id[B_THREADS];
    __shared__ float4 s_xy[B_THREADS];
    __shared__ float4 s_co[B_THREADS];
    grid_dependency_wait();
    __shared__ float4 s_rgb[B_THREADS];
    __shared__ int s_last;
    const int tile = blockIdx.x;
    const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
    const int x0 = tx * a.cam.tw, y0 = ty * a.cam.th;
    const int lxi = threadIdx.x & (a.cam.tw - 1), lyi = threadIdx.x >> a.cam.tw_log2;
    const int px = x0 + lxi, py = y0 + lyi;
    const int W = a.cam.W, H = a.cam.H;
    const bool inside = px < W && py < H;
    const float fx = (float)lxi, fy = (float)lyi; // pixel in the tile
    const uint2 range = a.ranges[tile];
    if (threadIdx.x == 0) s_last = -1;

    // 1) forward replay: final transmittance and the last blended pair of this pixel
    bool done = !inside;
    float T = 1.0f;
    int last = -1;
    for (unsigned start = range.x; start < range.y; start += B_THREADS) {
        if (__syncthreads_count(!done) == 0) break;
        const unsigned j = start + threadIdx.x;
        if (j < range.y) {
            unsigned id = a.vals[j];
            if (id >= (unsigned long long)a.n) id = 0;
            const float4 m = a.mean2[id];
            s_xy[threadIdx.x] = make_float4(m.x - (float)x0, m.y, m.z - (float)y0, m.w);
            s_co[threadIdx.x] = a.quad[id];
        }
        __syncthreads();
        const int cnt = min((unsigned)B_THREADS, range.y - start);
        for (int k = 0; !done && k < cnt; k++) {
            float dx, dy, e, alpha;
            if (!exact_alpha(s_xy[k], s_co[k], fx, fy, dx, dy, e, alpha)) continue;
            const float Tn = T * (1.0f - alpha);
            if (Tn < 1e-4f) {
                done = true;
                continue;
            }
            T = Tn;
            last = (int)(start + k);
        }
    }
    __syncthreads();
    if (last >= 0) atomicMax(&s_last, last);
    float G[3] = {0.f, 0.f, 0.f};
    if (inside) {
        const size_t plane = (size_t)W * H, o = (size_t)py * W + px;
        G[0] = a.dL_dimg[o];
        G[1] = a.dL_dimg[plane + o];
        G[2] = a.dL_dimg[2 * plane + o];
    }
    __syncthreads();
    const int block_last = s_last;
    if (block_last < 0) return;

    // 2) back to front over the same pairs
    float R[3] = {a.cam.bg[0] * T, a.cam.bg[1] * T, a.cam.bg[2] * T};
    const unsigned first_batch = range.x + (((unsigned)block_last - range.x) / B_THREADS) * B_THREADS;
    const int lane = threadIdx.x & 31;
    for (long long start = first_batch; start >= (long long)range.x; start -= B_THREADS) {
        __syncthreads();
        const unsigned j = (unsigned)start + threadIdx.x;
        if (j < range.y) {
            unsigned id = a.vals[j];
            if (id >= (unsigned long long)a.n) id = 0;
            s_id[threadIdx.x] = id;
            const float4 m = a.mean2[id];
            s_xy[threadIdx.x] = make_float4(m.x - (float)x0, m.y, m.z - (float)y0, m.w);
            s_co[threadIdx.x] = a.quad[id];
            s_rgb[threadIdx.x] = make_float4(a.rgb[3 * id], a.rgb[3 * id + 1], a.rgb[3 * id + 2], 0.f);
        }
        __syncthreads();
        const int cnt = min((long long)B_THREADS, (long long)range.y - start);
        for (int k = cnt - 1; k >= 0; k--) {
            const int jj = (int)start + k;
            float g_u = 0.f, g_v = 0.f, g_a = 0.f, g_b = 0.f, g_c = 0.f, g_o = 0.f, g_r = 0.f, g_g = 0.f, g_bl = 0.f;
            bool act = false;
            if (jj <= last) {
                float dx, dy, e, alpha;
                const float4 qd = s_co[k];
                if (exact_alpha(s_xy[k], qd, fx, fy, dx, dy, e, alpha)) {
                    // the conic (A, B, C) = Sigma'^-1 of the completed-square coefficients
                    const float cA = -2.0f * qd.x, cB = 2.0f * qd.x * qd.y;
                    const float4 co = make_float4(cA, cB, fmaf(-cB, qd.y, -2.0f * qd.z), qd.w);
                    act = true;
                    const float4 c = s_rgb[k];
                    const float inv = 1.0f / (1.0f - alpha);
                    const float Ti = T * inv;
                    const float wgt = alpha * Ti;
                    g_r = G[0] * wgt;
                    g_g = G[1] * wgt;
                    g_bl = G[2] * wgt;
                    const float dal = G[0] * (c.x * Ti - R[0] * inv) + G[1] * (c.y * Ti - R[1] * inv) +
                                      G[2] * (c.z * Ti - R[2] * inv);
                    R[0] += c.x * wgt;
                    R[1] += c.y * wgt;
                    R[2] += c.z * wgt;
                    T = Ti;
                    const bool clamped = co.w * e > 0.99f;
                    const float dpow = clamped ? 0.f : dal * alpha;
                    g_o = clamped ? 0.f : dal * e;
                    // power = -0.5 (A dx^2 + C dy^2) - B dx dy, dx = u - x, dy = v - y
                    g_u = -dpow * (co.x * dx + co.y * dy);
                    g_v = -dpow * (co.z * dy + co.y * dx);
                    g_a = -0.5f * dpow * dx * dx;
                    g_b = -dpow * dx * dy;
                    g_c = -0.5f * dpow * dy * dy;
                }
            }
            if (__any_sync(0xffffffffu, act)) {
                g_u = warp_red(g_u);
                g_v = warp_red(g_v);
                g_a = warp_red(g_a);
                g_b = warp_red(g_b);
                g_c = warp_red(g_c);
                g_o = warp_red(g_o);
                g_r = warp_red(g_r);
                g_g = warp_red(g_g);
                g_bl = warp_red(g_bl);
                if (lane == 0) {
                    float* g = a.gbuf + (size_t)s_id[k] * 9;
                    atomicAdd(g + 0, g_u);
                    atomicAdd(g + 1, g_v);
                    atomicAdd(g + 2, g_a);
                    atomicAdd(g + 3, g_b);
                    atomicAdd(g + 4, g_c);
                    atomicAdd(g + 5, g_o);
                    atomicAdd(g + 6, g_r);
                    atomicAdd(g + 7, g_g);
                    atomicAdd(g + 8, g_bl);
                }
            }
        }
    }
}

// gradient of the real SH basis (polynomial form; the tangential projection of the
// view direction removes the normal component)
__device__ __forceinline__ void sh_basis_grad(float x, float y, float z, float gx[16], float gy[16], float gz[16])
{
    const float k1 = 0.4886025119029199f, k2a = 1.0925484305920792f, k20 = 0.31539156525252005f;
    const float k22 = 0.5462742152960396f, k33 = 0.5900435899266435f, k32 = 2.890611442640554f;
    const float k31 = 0.4570457994644658f, k30 = 0.3731763325901154f, k32b = 1.445305721320277f;
    for (int k = 0; k < 16; k++) gx[k] = gy[k] = gz[k] = 0.f;
    gy[1] = k1;
    gz[2] = k1;
    gx[3] = k1;
    gx[4] = k2a * y; gy[4] = k2a * x;
    gy[5] = k2a * z; gz[5] = k2a * y;
    gz[6] = 6.f * k20 * z;
    gx[7] = k2a * z; gz[7] = k2a * x;
    gx[8] = 2.f * k22 * x; gy[8] = -2.f * k22 * y;
    gx[9] = 6.f * k33 * x * y; gy[9] = 3.f * k33 * (x * x - y * y);
    gx[10] = k32 * y * z; gy[10] = k32 * x * z; gz[10] = k32 * x * y;
    gy[11] = k31 * (5.f * z * z - 1.f); gz[11] = 10.f * k31 * y * z;
    gz[12] = k30 * (15.f * z * z - 3.f);
    gx[13] = k31 * (5.f * z * z - 1.f); gz[13] = 10.f * k31 * x * z;
    gx[14] = 2.f * k32b * x * z; gy[14] = -2.f * k32b * y * z; gz[14] = k32b * (x * x - y * y);
    gx[15] = 3.f * k33 * (x * x - y * y); gy[15] = -6.f * k33 * x * y;
}

__global__ void __launch_bounds__(128) k_preprocess_backward(BackwardArgs a)
{
    grid_dependency_wait();
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    float* dm = a.dmeans + 3 * i;
    float* ds = a.dscales + 3 * i;
    float* dq = a.dquats + 4 * i;
    float* dsh = a.dsh + 48 * i;
    for (int k = 0; k < 3; k++) dm[k] = ds[k] = 0.f;
    for (int k = 0; k < 4; k++) dq[k] = 0.f;
    for (int k = 0; k < 48; k++) dsh[k] = 0.f;
    a.dopac[i] = 0.f;
    if (a.touched[i] == 0) return; // emitted no entry: no pixel depends on it
    const float* g = a.gbuf + 9 * i;
    const float g_u = g[0], g_v = g[1], g_A = g[2], g_B = g[3], g_C = g[4];
    a.dopac[i] = g[5];
    const CamDev& c = a.cam;
    const float mx = a.means[3 * i], my = a.means[3 * i + 1], mz = a.means[3 * i + 2];
    const float s[3] = {a.scales[3 * i], a.scales[3 * i + 1], a.scales[3 * i + 2]};
    const float4 q4 = *reinterpret_cast<const float4*>(a.quats + 4 * i);
    const float qr[4] = {q4.x, q4.y, q4.z, q4.w};
    float p[3];
    for (int r = 0; r < 3; r++) p[r] = c.R[3 * r] * mx + c.R[3 * r + 1] * my + c.R[3 * r + 2] * mz + c.t[r];
    const float qnorm = sqrtf(qr[0] * qr[0] + qr[1] * qr[1] + qr[2] * qr[2] + qr[3] * qr[3]);
    const float w = qr[0] / qnorm, x = qr[1] / qnorm, y = qr[2] / qnorm, z = qr[3] / qnorm;
    float Q[9];
    Q[0] = 1.f - 2.f * (y * y + z * z); Q[1] = 2.f * (x * y - w * z);     Q[2] = 2.f * (x * z + w * y);
    Q[3] = 2.f * (x * y + w * z);     Q[4] = 1.f - 2.f * (x * x + z * z); Q[5] = 2.f * (y * z - w * x);
    Q[6] = 2.f * (x * z - w * y);     Q[7] = 2.f * (y * z + w * x);     Q[8] = 1.f - 2.f * (x * x + y * y);
    float M[9];
    for (int r = 0; r < 3; r++)
        for (int k = 0; k < 3; k++) M[3 * r + k] = Q[3 * r + k] * s[k];
    const float iz = 1.0f / p[2];
    const float xz = p[0] * iz, yz = p[1] * iz;
    const bool inx = xz > -c.limx && xz < c.limx, iny = yz > -c.limy && yz < c.limy;
    const float cxz = fminf(c.limx, fmaxf(-c.limx, xz)), cyz = fminf(c.limy, fmaxf(-c.limy, yz));
    const float J00 = c.fx * iz, J02 = -c.fx * cxz * iz, J11 = c.fy * iz, J12 = -c.fy * cyz * iz;
    float A2[6];
    for (int k = 0; k < 3; k++) {
        A2[k] = J00 * c.R[k] + J02 * c.R[6 + k];
        A2[3 + k] = J11 * c.R[3 + k] + J12 * c.R[6 + k];
    }
    float U[6];
    for (int r = 0; r < 2; r++)
        for (int k = 0; k < 3; k++)
            U[3 * r + k] = A2[3 * r] * M[k] + A2[3 * r + 1] * M[3 + k] + A2[3 * r + 2] * M[6 + k];
    const float sa = U[0] * U[0] + U[1] * U[1] + U[2] * U[2] + 0.3f;
    const float sc = U[3] * U[3] + U[4] * U[4] + U[5] * U[5] + 0.3f;
    const float sb = U[0] * U[3] + U[1] * U[4] + U[2] * U[5];
    // det Sigma' by the Lagrange identity |U0 x U1|^2 + 0.3 (|U0|^2 + |U1|^2) + 0.09, as the
    // forward computes it (sa sc - sb^2 cancels for thin Gaussians)
    const float x0 = U[1] * U[5] - U[2] * U[4], x1 = U[2] * U[3] - U[0] * U[5], x2 = U[0] * U[4] - U[1] * U[3];
    const float det = x0 * x0 + x1 * x1 + x2 * x2 + 0.3f * (sa + sc - 0.6f) + 0.09f;
    const float idet = 1.0f / det;
    // K = Sigma'^-1 = [[A, B], [B, C]]; dL/dSigma' = -K Gs K with Gs = [[gA, gB/2], [gB/2, gC]]
    const float KA = sc * idet, KB = -sb * idet, KC = sa * idet;
    const float G00 = g_A, G01 = 0.5f * g_B, G11 = g_C;
    const float t00 = KA * G00 + KB * G01, t01 = KA * G01 + KB * G11;
    const float t10 = KB * G00 + KC * G01, t11 = KB * G01 + KC * G11;
    const float H00 = -(t00 * KA + t01 * KB), H01 = -(t00 * KB + t01 * KC), H11 = -(t10 * KB + t11 * KC);
    // dL/dU = 2 H U
    float dU[6];
    for (int k = 0; k < 3; k++) {
        dU[k] = 2.f * (H00 * U[k] + H01 * U[3 + k]);
        dU[3 + k] = 2.f * (H01 * U[k] + H11 * U[3 + k]);
    }
    // U = A2 M: dA2 = dU M^T, dM = A2^T dU
    float dA2[6], dM[9];
    for (int r = 0; r < 2; r++)
        for (int k = 0; k < 3; k++)
            dA2[3 * r + k] = dU[3 * r] * M[3 * k] + dU[3 * r + 1] * M[3 * k + 1] + dU[3 * r + 2] * M[3 * k + 2];
    for (int r = 0; r < 3; r++)
        for (int k = 0; k < 3; k++) dM[3 * r + k] = A2[r] * dU[k] + A2[3 + r] * dU[3 + k];
    // M = Q diag(s)
    float dQ[9];
    for (int k = 0; k < 3; k++) ds[k] = dM[k] * Q[k] + dM[3 + k] * Q[3 + k] + dM[6 + k] * Q[6 + k];
    for (int r = 0; r < 3; r++)
        for (int k = 0; k < 3; k++) dQ[3 * r + k] = dM[3 * r + k] * s[k];
    // rotation of the unit quaternion (w, x, y, z)
    float dqn[4];
    dqn[0] = 2.f * (-z * dQ[1] + y * dQ[2] + z * dQ[3] - x * dQ[5] - y * dQ[6] + x * dQ[7]);
    dqn[1] = 2.f * (y * dQ[1] + z * dQ[2] + y * dQ[3] - 2.f * x * dQ[4] - w * dQ[5] + z * dQ[6] + w * dQ[7] -
                    2.f * x * dQ[8]);
    dqn[2] = 2.f * (-2.f * y * dQ[0] + x * dQ[1] + w * dQ[2] + x * dQ[3] + z * dQ[5] - w * dQ[6] + z * dQ[7] -
                    2.f * y * dQ[8]);
    dqn[3] = 2.f * (-2.f * z * dQ[0] - w * dQ[1] + x * dQ[2] + w * dQ[3] - 2.f * z * dQ[4] + y * dQ[5] + x * dQ[6] +
                    y * dQ[7]);
    const float qn[4] = {w, x, y, z};
    const float dotq = qn[0] * dqn[0] + qn[1] * dqn[1] + qn[2] * dqn[2] + qn[3] * dqn[3];
    for (int k = 0; k < 4; k++) dq[k] = (dqn[k] - qn[k] * dotq) / qnorm;
    // A2 = J W: dJ = dA2 W^T (only the four non-zero entries of J)
    const float dJ00 = dA2[0] * c.R[0] + dA2[1] * c.R[1] + dA2[2] * c.R[2];
    const float dJ02 = dA2[0] * c.R[6] + dA2[1] * c.R[7] + dA2[2] * c.R[8];
    const float dJ11 = dA2[3] * c.R[3] + dA2[4] * c.R[4] + dA2[5] * c.R[5];
    const float dJ12 = dA2[3] * c.R[6] + dA2[4] * c.R[7] + dA2[5] * c.R[8];
    float dp[3];
    const float iz2 = iz * iz;
    dp[0] = g_u * c.fx * iz + (inx ? dJ02 * (-c.fx * iz2) : 0.f);
    dp[1] = g_v * c.fy * iz + (iny ? dJ12 * (-c.fy * iz2) : 0.f);
    dp[2] = -g_u * c.fx * p[0] * iz2 - g_v * c.fy * p[1] * iz2 - dJ00 * c.fx * iz2 - dJ11 * c.fy * iz2 +
            dJ02 * (inx ? 2.f * c.fx * p[0] * iz2 * iz : c.fx * cxz * iz2) +
            dJ12 * (iny ? 2.f * c.fy * p[1] * iz2 * iz : c.fy * cyz * iz2);
    for (int k = 0; k < 3; k++) dm[k] = c.R[k] * dp[0] + c.R[3 + k] * dp[1] + c.R[6 + k] * dp[2];
    // colour = clamp(sum_k Y_k(d) SH_k + 0.5)
    const float vx = mx - c.campos[0], vy = my - c.campos[1], vz = mz - c.campos[2];
    const float vn = sqrtf(vx * vx + vy * vy + vz * vz);
    const float dx = vx / vn, dy = vy / vn, dz = vz / vn;
    float Y[16], gx[16], gy[16], gz[16];
    sh_basis(dx, dy, dz, Y);
    sh_basis_grad(dx, dy, dz, gx, gy, gz);
    const int nk = (a.sh_degree + 1) * (a.sh_degree + 1);
    const float* sh = a.sh + 48 * i;
    float gd[3] = {0.f, 0.f, 0.f};
    for (int ch = 0; ch < 3; ch++) {
        float raw = 0.5f;
        for (int k = 0; k < nk; k++) raw += Y[k] * sh[3 * k + ch];
        if (!(raw > 0.0f && raw < 1.0f)) continue; // clamped channel
        const float gc = g[6 + ch];
        for (int k = 0; k < nk; k++) {
            dsh[3 * k + ch] = Y[k] * gc;
            gd[0] += gc * sh[3 * k + ch] * gx[k];
            gd[1] += gc * sh[3 * k + ch] * gy[k];
            gd[2] += gc * sh[3 * k + ch] * gz[k];
        }
    }
    const float dd = gd[0] * dx + gd[1] * dy + gd[2] * dz; // tangential part / |v|
    dm[0] += (gd[0] - dd * dx) / vn;
    dm[1] += (gd[1] - dd * dy) / vn;
    dm[2] += (gd[2] - dd * dz) / vn;
}

void launch_raster_backward(const BackwardArgs& a, cudaStream_t s)
{
    const unsigned tiles = (unsigned)(a.tiles_x * a.tiles_y);
    launch_dependent(k_raster_backward, dim3(tiles), dim3(B_THREADS), 0, s, a);
}

void launch_preprocess_backward(const BackwardArgs& a, cudaStream_t s)
{
    if (a.n <= 0) return;
    launch_dependent(k_preprocess_backward, dim3((unsigned)((a.n + 127) / 128)), dim3(128), 0, s, a);
}

} // namespace rg
