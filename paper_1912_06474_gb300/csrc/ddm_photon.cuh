// Photon mapping through the domain decomposition (Sec. 4 photon mapping,
// Sec. 5 sub-domains). Included by ddm.cu: it reuses the ray queues, the
// scatter and the trace kernel unchanged.
//
// Photon pass: k_photon_emit starts photon i at a point of the area lights
// (triangle by area, uniform point, cosine direction about the front face,
// power pi Le A / N) and stages its ray in the queue of the subdomain where it
// enters the grid; every hit b = 1 .. D-1 runs the subdomain waves, then
// k_photon_shade stores the photon at a diffuse hit once a bounce or a
// reflection has changed its direction and continues it like a camera path
// (diffuse bounce times rho, conductor mirror times Fresnel, glass branch with
// R/P, T/(1-P)). The photon's power lives in the path state's throughput rows.
// Philox counter (photon, 0xffffffff, hit, slot), key (seed, render id).
//
// Camera pass: k_ddm_gather adds, at a path's diffuse vertex, the power of
// the photons within radius r on the visible side times rho / pi / (pi r^2);
// k_shade_continue then issues the shadow ray but no continuation.

constexpr int kFlPhotonTurned = 16;   // the photon's direction has changed (bounce or reflection)
constexpr int kFlPhotonDiffuse = 32;  // ... by a diffuse bounce (else it is a caustic photon)

struct PhotonPass {
    int64_t begin, n_total;
    int max_depth;
    uint32_t seed, render_id;
    float scale;                // pi * total light area / n_total
    const float *state_s;
    float4 *pos, *dir;
    float *pow;
};

__global__ void __launch_bounds__(256) k_photon_emit(KArgs a, PhotonPass pp) {
    const int64_t np = a.ps.np;
    const DevScene &sc = a.sc;
    const int L = sc.L;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long n_ext = 0;
    __shared__ PushSmem psm;
    int *bins = block_bins_init(a.g.n_bins);
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < np; base += stride) {   // block-uniform trips
        const int64_t q = base + threadIdx.x;
        bool want = false;
        int cell = 0;
        float4 r0 = make_float4(0, 0, 0, 0), r1 = r0;
        int4 r2 = make_int4(0, 0, 0, 0);
        if (q < np) {
            a.ps.flags[q] = 0;
            if (sc.n_light > 0) {
                const uint32_t pi = (uint32_t)(pp.begin + q), pj = 0xffffffffu;
                uint4 xl = philox4x32_10(make_uint4(pi, pj, 0u, kSlotLight), pp.seed, pp.render_id);
                const float ua = u01(xl.x), su = sqrtf(u01(xl.y)), u2 = u01(xl.z);
                int li = sc.n_light - 1;
                for (int k = 0; k < sc.n_light; ++k)
                    if (ua < __ldg(sc.light_cdf + k)) { li = k; break; }
                const float4 lv0 = __ldg(sc.light_v + 3 * li), lv1 = __ldg(sc.light_v + 3 * li + 1),
                             lv2 = __ldg(sc.light_v + 3 * li + 2);
                const int lt = __float_as_int(lv0.w);
                const float4 ln = __ldg(sc.tri_n + lt);
                const V3 nl = xyz(ln);
                const float b0 = 1.0f - su, b1 = u2 * su, b2 = 1.0f - b0 - b1;
                const V3 o = b0 * xyz(lv0) + b1 * xyz(lv1) + b2 * xyz(lv2) + kRayOffset * nl;
                uint4 xd = philox4x32_10(make_uint4(pi, pj, 0u, kSlotBsdf), pp.seed, pp.render_id);
                const V3 d = cosine_dir(nl, u01(xd.x), u01(xd.y));
                const float *Le = sc.mat_a + (size_t)__float_as_int(ln.w) * L;
                for (int i = 0; i < L; ++i) a.ps.T[(size_t)i * np + q] = __ldg(Le + i) * pp.scale;
                a.ps.flags[q] = kFlExt;
                a.ps.hit0[q] = make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
                ++n_ext;
                float t0;
                if (grid_enter(a.g, o, d, __int_as_float(0x7f800000), t0, cell)) {
                    want = true;
                    r0 = make_float4(o.x, o.y, o.z, t0);
                    r1 = make_float4(d.x, d.y, d.z, __int_as_float(0x7f800000));
                    r2 = make_int4((int)q, lt, 0, cell);
                }
            }
        }
        block_stage_push2(a.Q, a.g, psm, bins, want, cell, r0, r1, r2, false, 0, r0, r1, r2, a.err);
    }
    block_bins_flush(a.Q, bins, a.g.n_bins);
    block_count3(a.counters + 0, n_ext, nullptr, 0, nullptr, 0);
}

// Power rows of the photons a warp stores are written row by row by the whole
// warp (coalesced) through a [L][33] shared-memory tile per warp, for L up to
// kStageMaxL; one lane per row otherwise.
constexpr int kStageMaxL = 64;
__host__ __device__ constexpr size_t photon_stage_bytes(int L) {
    return L <= kStageMaxL ? (size_t)8 * L * 33 * sizeof(float) : 0;
}

template <bool FILMS>
__global__ void __launch_bounds__(256) k_photon_shade(KArgs a, PhotonPass pp) {
    const int64_t np = a.ps.np;
    const DevScene &sc = a.sc;
    const int L = sc.L, b = a.b, D = pp.max_depth;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long n_ext = 0;
    __shared__ PushSmem psm;
    int *bins = block_bins_init(a.g.n_bins);
    const bool staged = L <= kStageMaxL;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float *stage = reinterpret_cast<float *>(bins + ((a.g.n_bins + 3) & ~3)) + (size_t)w * L * 33;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < np; base += stride) {   // block-uniform trips
        const int64_t q = base + threadIdx.x;
        bool want = false;
        int cell = 0;
        float4 e0 = make_float4(0, 0, 0, 0), e1 = e0;
        int4 e2 = make_int4(0, 0, 0, 0);
        const int fl = q < np ? a.ps.flags[q] : 0;
        if (staged) {
            bool store = false;
            if ((fl & kFlExt) && (fl & kFlPhotonTurned)) {
                const int prim = __float_as_int(a.ps.hit0[q].w);
                if (prim >= 0) {
                    const int kind = __ldg(sc.mat_kind + __float_as_int(__ldg(sc.tri_n + prim).w));
                    store = kind == kLambert || kind == kDiffuseEmitter;
                }
            }
            const unsigned sm = __ballot_sync(0xffffffffu, store);
            if (sm) {
                if (store)
                    for (int i = 0; i < L; ++i) stage[i * 33 + lane] = a.ps.T[(size_t)i * np + q];
                __syncwarp();
                for (unsigned m = sm; m; m &= m - 1) {
                    const int src = __ffs(m) - 1;
                    const size_t slot = (size_t)(pp.begin + base + 32 * w + src) * (D - 1) + (b - 1);
                    for (int i = lane; i < L; i += 32) pp.pow[slot * L + i] = stage[i * 33 + src];
                }
                __syncwarp();
            }
        }
        if (fl & kFlExt) {
            int nfl = 0;
            const float4 h0 = a.ps.hit0[q], h1 = a.ps.hit1[q];
            const int prim = __float_as_int(h0.w);
            if (prim >= 0) {
                const uint32_t pi = (uint32_t)(pp.begin + q), pj = 0xffffffffu;
                const float4 tn = __ldg(sc.tri_n + prim);
                const V3 ng = xyz(tn), x = xyz(h0), d = xyz(h1);
                const int mat = __float_as_int(tn.w), kind = __ldg(sc.mat_kind + mat);
                const float cd = dot(d, ng);
                const V3 ns = cd < 0.0f ? ng : (-1.0f) * ng;
                const float *mA = sc.mat_a + (size_t)mat * L, *mB = sc.mat_b + (size_t)mat * L;
                bool go = false, turn = true, diffuse = false;   // a transmitted photon keeps its direction
                V3 on = x, dn = d;
                int excl = prim;
                if (kind == kLambert || kind == kDiffuseEmitter) {
                    if (fl & kFlPhotonTurned) {
                        const size_t slot = (size_t)(pp.begin + q) * (D - 1) + (b - 1);
                        // w: 1 global photon, 2 caustic photon (only reflections turned it)
                        pp.pos[slot] = make_float4(x.x, x.y, x.z, (fl & kFlPhotonDiffuse) ? 1.0f : 2.0f);
                        pp.dir[slot] = make_float4(d.x, d.y, d.z, 0.0f);
                        if (!staged) {
                            float *pw = pp.pow + slot * L;
                            for (int i = 0; i < L; ++i) pw[i] = a.ps.T[(size_t)i * np + q];
                        }
                    }
                    if (b < D - 1) {
                        const float *rho = kind == kLambert ? mA : mB;
                        uint4 xb = philox4x32_10(make_uint4(pi, pj, (uint32_t)b, kSlotBsdf), pp.seed, pp.render_id);
                        dn = cosine_dir(ns, u01(xb.x), u01(xb.y));
                        for (int i = 0; i < L; ++i) a.ps.T[(size_t)i * np + q] *= __ldg(rho + i);
                        on = x + kRayOffset * ns;
                        go = true;
                        diffuse = true;
                    }
                } else if (kind == kConductor) {
                    if (b < D - 1) {
                        const float c = fabsf(cd);
                        for (int i = 0; i < L; ++i)
                            a.ps.T[(size_t)i * np + q] *= conductor_F(c, __ldg(mA + i), __ldg(mB + i));
                        dn = d - (2.0f * cd) * ng;
                        on = x + kRayOffset * ns;
                        go = true;
                    }
                } else if (kind == kGlass) {
                    if (b < D - 1) {
                        const float c = fabsf(cd);
                        const float pr = branch_proxy(c, L, mA);
                        uint4 xg = philox4x32_10(make_uint4(pi, pj, (uint32_t)b, kSlotGlass), pp.seed, pp.render_id);
                        const bool refl = u01(xg.x) < pr;
                        const float st = __ldg(pp.state_s + mat), th = __ldg(sc.mat_thick + mat);
                        const float wsel = refl ? 1.0f / pr : 1.0f / (1.0f - pr);
                        for (int i = 0; i < L; ++i) {
                            float R_, T_;
                            glass_rt<FILMS>(sc, mat, i, c, st, th, R_, T_);
                            a.ps.T[(size_t)i * np + q] *= (refl ? R_ : T_) * wsel;
                        }
                        if (refl) {
                            dn = d - (2.0f * cd) * ng;
                            on = x + kRayOffset * ns;
                        } else {
                            on = x - kRayOffset * ns;
                            excl = -__ldg(sc.tri_obj + prim) - 2;
                            turn = false;
                        }
                        go = true;
                    }
                }
                if (go) {
                    nfl = kFlExt | ((turn || (fl & kFlPhotonTurned)) ? kFlPhotonTurned : 0) |
                          ((diffuse || (fl & kFlPhotonDiffuse)) ? kFlPhotonDiffuse : 0);
                    ++n_ext;
                    a.ps.hit0[q] = make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
                    float t0;
                    if (grid_enter(a.g, on, dn, __int_as_float(0x7f800000), t0, cell)) {
                        want = true;
                        e0 = make_float4(on.x, on.y, on.z, t0);
                        e1 = make_float4(dn.x, dn.y, dn.z, __int_as_float(0x7f800000));
                        e2 = make_int4((int)q, excl, 0, cell);
                    }
                }
            }
            a.ps.flags[q] = nfl;
        }
        block_stage_push2(a.Q, a.g, psm, bins, want, cell, e0, e1, e2, false, 0, e0, e1, e2, a.err);
    }
    block_bins_flush(a.Q, bins, a.g.n_bins);
    block_count3(a.counters + 0, n_ext, nullptr, 0, nullptr, 0);
}

// Photon-map radiance at the diffuse vertex of each path of this bounce.
__global__ void __launch_bounds__(256) k_ddm_gather(KArgs a) {
    const int64_t np = a.ps.np;
    const DevScene &sc = a.sc;
    const int L = sc.L, b = a.b;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const PathState &ps = a.ps;
    // rho / pi times the power over pi r^2 of each map (global, caustic)
    const float inv_g = 1.0f / (3.14159265358979f * a.pm.radius * a.pm.radius);
    const float inv_c = a.pmc.on ? 1.0f / (3.14159265358979f * a.pmc.radius * a.pmc.radius) : 0.0f;
    const float norm = 1.0f / 3.14159265358979f;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < np; q += stride) {
        const int fl = ps.flags[q];
        if (!(fl & kFlExt)) continue;
        const RenderInfo &ri = a.rb.info[find_render(a.rb, a.path_begin + q)];
        if (b > ri.max_depth) continue;
        const float4 h0 = ps.hit0[q];
        const int prim = __float_as_int(h0.w);
        if (prim < 0) continue;
        const float4 tn = __ldg(sc.tri_n + prim);
        const int mat = __float_as_int(tn.w), kind = __ldg(sc.mat_kind + mat);
        if (kind != kLambert && kind != kDiffuseEmitter) continue;
        const V3 ng = xyz(tn), d = xyz(ps.hit1[q]);
        const V3 ns = dot(d, ng) < 0.0f ? ng : (-1.0f) * ng;
        float S[kMaxL];
        for (int i = 0; i < L; ++i) S[i] = 0.0f;
        pm_gather_visit(a.pm, xyz(h0), ns, [&](int slot) {
            const float *pw = a.pm.pow + (size_t)slot * L;
            for (int i = 0; i < L; ++i) S[i] += __ldg(pw + i);
        });
        for (int i = 0; i < L; ++i) S[i] *= inv_g;
        if (a.pmc.on)
            pm_gather_visit(a.pmc, xyz(h0), ns, [&](int slot) {
                const float *pw = a.pmc.pow + (size_t)slot * L;
                for (int i = 0; i < L; ++i) S[i] = fmaf(__ldg(pw + i), inv_c, S[i]);
            });
        const float *rho = (kind == kLambert ? sc.mat_a : sc.mat_b) + (size_t)mat * L;
        Kahan X, Y, Z;
        for (int i = 0; i < L; ++i) {
            const float e = ps.T[(size_t)i * np + q] * __ldg(rho + i) * S[i] * norm;
            const float4 w4 = __ldg(sc.wcmf + i);
            X.add(e * w4.x);
            Y.add(e * w4.y);
            Z.add(e * w4.z);
        }
        Kahan3 acc;
        acc.x.s = ps.acc[0 * np + q];
        acc.y.s = ps.acc[1 * np + q];
        acc.z.s = ps.acc[2 * np + q];
        acc.x.c = ps.acc[3 * np + q];
        acc.y.c = ps.acc[4 * np + q];
        acc.z.c = ps.acc[5 * np + q];
        acc.add(X.s, Y.s, Z.s);
        ps.acc[0 * np + q] = acc.x.s;
        ps.acc[1 * np + q] = acc.y.s;
        ps.acc[2 * np + q] = acc.z.s;
        ps.acc[3 * np + q] = acc.x.c;
        ps.acc[4 * np + q] = acc.y.c;
        ps.acc[5 * np + q] = acc.z.c;
    }
}

int ddm_photon_pass(const DDMPhotonRun &run, DDMBuffers &buf, cudaStream_t s) {
    const int64_t np = run.count;
    const int L = run.sc.L;
    const int nb = run.g.n_bins;
    if (run.g.n_cells > kMaxCells || nb > kMaxBins) {
        set_error("sddm_render_photon_map: the DDM method supports at most 2048 subdomains");
        return SDDM_ERR_INVALID_ARG;
    }
    if (np <= 0 || run.max_depth < 2) return SDDM_OK;
    const int64_t cap = np;   // one ray per photon in flight
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = (off + bytes + 255) & ~(size_t)255;
        return o;
    };
    const size_t oT = take(sizeof(float) * (size_t)L * np), oFl = take(4 * np), oH0 = take(16 * np),
                 oH1 = take(16 * np), oIn = take(48 * cap), oSt = take(48 * cap), oCtl = take(32 + 4 * (size_t)nb),
                 oFill = take(4 * (size_t)nb), oOff = take(4 * ((size_t)nb + 1));
    if (off > buf.bytes) {
        if (buf.mem) cudaFree(buf.mem);
        buf.mem = nullptr;
        buf.bytes = 0;
        cudaError_t e = cudaMalloc(&buf.mem, off);
        if (e != cudaSuccess) {
            buf.mem = nullptr;
            set_error("sddm_render_photon_map: photon-state allocation failed");
            return SDDM_ERR_OOM;
        }
        buf.bytes = off;
    }
    char *m = (char *)buf.mem;
    KArgs a{};
    a.sc = run.sc;
    a.g = run.g;
    a.counters = run.counters;
    a.err = run.error_flag;
    a.ps.np = np;
    a.ps.T = (float *)(m + oT);
    a.ps.flags = (int *)(m + oFl);
    a.ps.hit0 = (float4 *)(m + oH0);
    a.ps.hit1 = (float4 *)(m + oH1);
    Queues &Q = a.Q;
    Q.cap = cap;
    Q.in = (float4 *)(m + oIn);
    Q.stage = (float4 *)(m + oSt);
    Q.ctl = (unsigned long long *)(m + oCtl);
    Q.cnt = (int *)(m + oCtl + 32);
    Q.fill = (int *)(m + oFill);
    Q.off = (int *)(m + oOff);
    PhotonPass pp;
    pp.begin = run.begin;
    pp.n_total = run.n_total;
    pp.max_depth = run.max_depth;
    pp.seed = run.seed;
    pp.render_id = run.render_id;
    pp.scale = 3.14159265358979f * run.sc.light_area / (float)run.n_total;
    pp.state_s = run.state_s;
    pp.pos = run.pos;
    pp.dir = run.dir;
    pp.pow = run.pow;

    const int sm = std::max(1, run.sm_count);
    const unsigned path_blocks = (unsigned)std::min<int64_t>((np + 255) / 256, (int64_t)sm * 16);
    const int trace_blocks = sm * (run.blocks_per_sm > 0 ? run.blocks_per_sm : 8);
    const int scatter_blocks = sm * 4;
    const int waves = ddm_waves(run.g);
    const size_t ctl_bytes = 32 + 4 * (size_t)nb;
    const size_t bins_smem = sizeof(int) * (size_t)nb;
    cudaError_t e;
#define PM_CHECK(x)                                                                \
    do {                                                                           \
        if ((e = (x)) != cudaSuccess) return cuda_fail(e, "sddm_render_photon_map: " #x); \
    } while (0)
    PM_CHECK(cudaMemsetAsync(Q.ctl, 0, ctl_bytes, s));
    k_photon_emit<<<path_blocks, 256, bins_smem, s>>>(a, pp);
    PM_CHECK(cudaGetLastError());
    *run.launches += 1;
    for (int b = 1; b <= run.max_depth - 1; ++b) {
        for (int w = 0; w < waves; ++w) {
            PM_CHECK(cudaMemsetAsync(Q.fill, 0, 4 * (size_t)nb, s));
            k_scatter<<<scatter_blocks, 256, 0, s>>>(a);
            PM_CHECK(cudaGetLastError());
            PM_CHECK(cudaMemsetAsync(Q.ctl, 0, ctl_bytes, s));
            a.last_wave = w == waves - 1;
            a.g.continue_cells = ddm_wave_continues(run.g, w, waves);
            k_trace_wave<false><<<trace_blocks, 128, 0, s>>>(a);
            PM_CHECK(cudaGetLastError());
            *run.launches += 2;
        }
        a.b = b;
        const size_t shade_smem = sizeof(int) * (size_t)((nb + 3) & ~3) + photon_stage_bytes(L);
        if (run.sc.mat_nfilm) {
            PM_CHECK(cudaFuncSetAttribute(k_photon_shade<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)shade_smem));
            k_photon_shade<true><<<path_blocks, 256, shade_smem, s>>>(a, pp);
        } else {
            PM_CHECK(cudaFuncSetAttribute(k_photon_shade<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)shade_smem));
            k_photon_shade<false><<<path_blocks, 256, shade_smem, s>>>(a, pp);
        }
        PM_CHECK(cudaGetLastError());
        *run.launches += 1;
    }
#undef PM_CHECK
    return SDDM_OK;
}
