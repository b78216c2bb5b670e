// DDM trace kernel: one wave of closest-hit and shadow queries over the
// cell-sorted ray queue (Sec. 5's work inside one subdomain, with the
// interface hand-off to the neighbour). Included by ddm.cu after KArgs and
// the grid helpers; kept in its own file so that its source, which the
// recorded DRAM-traffic measurement belongs to, is identifiable.
#pragma once

// Distance at which the ray leaves `cell`, and the neighbour it enters
// (-1 when it leaves the grid). Ties between faces go x, then y, then z. The
// cell's planes and neighbours come from the per-cell table; distances use
// the ray's reciprocal direction.
__device__ __forceinline__ float cell_exit(const DDMScene &g, int cell, const Ray &r, int &next) {
    const float4 p0 = __ldg(g.cell_planes + 2 * cell), p1 = __ldg(g.cell_planes + 2 * cell + 1);
    const int4 n0 = __ldg(g.cell_next + 2 * cell), n1 = __ldg(g.cell_next + 2 * cell + 1);
    float t = __int_as_float(0x7f800000);
    next = -1;
    if (r.d.x != 0.0f) {
        const bool pos = r.d.x > 0.0f;
        const float ta = ((pos ? p0.y : p0.x) - r.o.x) * r.inv.x;
        if (ta < t) {
            t = ta;
            next = pos ? n0.y : n0.x;
        }
    }
    if (r.d.y != 0.0f) {
        const bool pos = r.d.y > 0.0f;
        const float ta = ((pos ? p0.w : p0.z) - r.o.y) * r.inv.y;
        if (ta < t) {
            t = ta;
            next = pos ? n0.w : n0.z;
        }
    }
    if (r.d.z != 0.0f) {
        const bool pos = r.d.z > 0.0f;
        const float ta = ((pos ? p1.y : p1.x) - r.o.z) * r.inv.z;
        if (ta < t) {
            t = ta;
            next = pos ? n1.y : n1.x;
        }
    }
    return t;
}

// Block-wide sums of up to three statistics counters, one atomic per counter
// and block. All threads of the block call it.
__device__ __forceinline__ void block_count3(unsigned long long *c0, unsigned long long v0, unsigned long long *c1,
                                             unsigned long long v1, unsigned long long *c2, unsigned long long v2) {
    __shared__ unsigned long long s_red[32][3];
    for (int off = 16; off > 0; off >>= 1) {
        v0 += __shfl_down_sync(0xffffffffu, v0, off);
        v1 += __shfl_down_sync(0xffffffffu, v1, off);
        v2 += __shfl_down_sync(0xffffffffu, v2, off);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        s_red[w][0] = v0;
        s_red[w][1] = v1;
        s_red[w][2] = v2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t0 = 0, t1 = 0, t2 = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            t0 += s_red[k][0];
            t1 += s_red[k][1];
            t2 += s_red[k][2];
        }
        if (c0 && t0) atomicAdd(c0, t0);
        if (c1 && t1) atomicAdd(c1, t1);
        if (c2 && t2) atomicAdd(c2, t2);
    }
}

// ------------------------------------------------------ trace one wave
// Persistent warps whose lanes are refilled one by one: a lane that finishes
// its ray (hit, occlusion, or exit from the cell) takes the next ray of the
// cell-sorted queue while the other lanes carry on, so a warp is not held by
// its slowest ray. Traversal is a resumable state machine; each round runs the
// warp through interior nodes until every lane stands at a leaf (at most
// kTraceSteps steps), then through the leaves, then refills.
#ifndef SDDM_TRACE_STEPS
#define SDDM_TRACE_STEPS 64   // interior steps per round at most
#endif
constexpr int kTraceSteps = SDDM_TRACE_STEPS;
// Queue slots a warp reserves per refill atomic (>= 32, so one run always covers a refill).
constexpr int kRefillChunk = 32;
// Rays a warp buffers in shared memory before appending them to the staging area.
constexpr int kPushBuf = 32;

// Append a warp's buffered rays to the staging area: one atomic, then the
// warp copies the 3 * n float4 words with consecutive lanes on consecutive words.
__device__ __forceinline__ void flush_push_buf(const Queues &Q, const float4 *buf, int n, int lane, int *err) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(Q.ctl + 0, (unsigned long long)n);
    base = __shfl_sync(0xffffffffu, base, 0);
    __syncwarp();
    if (base + (unsigned long long)n > (unsigned long long)Q.cap) {
        if (lane == 0) atomicCAS(err, 0, 1);
        return;
    }
    float4 *dst = Q.stage + 3 * base;
    for (int k = lane; k < 3 * n; k += 32) dst[k] = buf[k];
    __syncwarp();
}
// Resident 128-thread blocks per SM the trace kernel is compiled for (register budget).
#ifndef SDDM_TRACE_MIN_BLOCKS
#define SDDM_TRACE_MIN_BLOCKS 8
#endif

// First device check to fail records its code and two details in the error word.
__device__ __forceinline__ void trace_check_fail(int *err, int code, int x, int y) {
    if (atomicCAS(err, 0, code) == 0) {
        err[1] = x;
        err[2] = y;
    }
}

// CHECKED (the subdomain cache, whose cells move between loads): every root,
// child and leaf index is checked against the records the cache holds before
// it is read; a bad one is recorded (codes 8-10) and the ray is dropped.
template <bool COUNT, bool CHECKED = false>
__global__ void __launch_bounds__(128, SDDM_TRACE_MIN_BLOCKS) k_trace_wave(KArgs a) {
    const Queues &Q = a.Q;
    const DDMScene &g = a.g;
    // the rays of this launch: the whole wave, or one group's range of it
    // (the groups of cells resident together in the subdomain cache)
    const int q0 = a.q_end > 0 ? (int)a.q_begin : 0;
    const int total = (a.q_end > 0 ? (int)a.q_end : Q.off[g.n_bins]) - q0;
    if (total <= 0) return;
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    const int64_t np = a.ps.np;
    unsigned long long n_cross = 0, n_vis = 0, n_cont = 0;   // n_cont: crossings carried on by the lane
    TravCount tc;

    __shared__ float4 s_push[128 / 32][3 * kPushBuf];   // per-warp hand-off buffers
    float4 *pbuf = s_push[threadIdx.x >> 5];
    int nbuf = 0;              // rays in the warp's buffer (uniform)
    int idx = -1;              // queue index of this lane's ray, -1 = none
    bool exhausted = false;    // no ray left for this lane
    __shared__ unsigned long long s_run[128 / 32][2];    // per warp: reserved run [begin, end) of queue slots
    unsigned long long *run = s_run[threadIdx.x >> 5];
    if (lane == 0) run[0] = run[1] = 0;
    __syncwarp();
    Ray ray;
    float t_cur = 0.f, t_max = 0.f, t_exit = 0.f, tmin = 0.f, tw = 0.f;
    int q = 0, excl = -1, rfl = 0, next = -1, node = 0, sp = 0, best = -1, ep = -1, eo = -1, n_prev = 0;
    bool occ = false;
    Crossings cr;
    cr.n = 0;
    int stack[kStackSize];

    for (;;) {
        // 1. idle lanes take the next rays of the queue, from a run of
        //    kRefillChunk queue slots the warp reserves at a time (one atomic
        //    per run instead of one per refill)
        const bool need = idx < 0 && !exhausted;
        const unsigned m = __ballot_sync(full, need);
        if (m) {
            const unsigned want = __popc(m);
            const unsigned long long cbeg = run[0], cend = run[1];
            const unsigned long long avail = cend - cbeg;
            unsigned long long nb = 0;
            if (avail < want) {
                if (lane == 0) nb = atomicAdd(Q.ctl + 1, (unsigned long long)kRefillChunk);
                nb = __shfl_sync(full, nb, 0);
            }
            const unsigned rank = __popc(m & lt_mask);
            const unsigned long long mine = rank < avail ? cbeg + rank : nb + (rank - avail);
            __syncwarp();
            if (lane == 0) {
                if (avail >= want) {
                    run[0] = cbeg + want;
                } else {
                    run[0] = nb + (want - avail);
                    run[1] = nb + kRefillChunk;
                }
            }
            __syncwarp();
            if (need) {
                const unsigned long long my = mine;
                if (my < (unsigned long long)total) {
                    idx = q0 + (int)my;
                    const float4 *src = Q.in + 3 * (size_t)idx;
                    const float4 r0 = src[0], r1 = src[1], r2f = src[2];
                    q = __float_as_int(r2f.x);
                    excl = __float_as_int(r2f.y);
                    rfl = __float_as_int(r2f.z);
                    int cell = __float_as_int(r2f.w);
                    if (CHECKED && (q < 0 || q >= np || cell < 0 || cell >= g.n_cells)) {
                        trace_check_fail(a.err, 12, q, cell);
                        q = 0;
                        cell = 0;
                    }
                    ray = make_ray(xyz(r0), xyz(r1));
                    t_cur = r0.w;
                    t_max = r1.w;
                    t_exit = cell_exit(g, cell, ray, next);
                    tmin = fmaxf(0.0f, t_cur - g.eps);
                    node = __ldg(g.root + cell);
                    if (CHECKED && (node < 0 || node >= g.node_cap)) {
                        trace_check_fail(a.err, 8, cell, node);
                        node = ~0;   // an empty leaf: the ray ends here
                    }
                    sp = 0;
                    best = -1;
                    occ = false;
                    ++n_vis;
                    if (rfl & kRayShadow) {
                        tw = fminf(t_exit + g.eps, t_max);
                        cr.n = (rfl >> 1) & 7;
                        for (int k = 0; k < cr.n; ++k) cr.obj[k] = a.ps.cross_obj[k * np + q];
                        n_prev = cr.n;
                    } else {
                        tw = t_exit + g.eps;
                        ep = excl >= 0 ? excl : -1;
                        eo = excl <= -2 ? -excl - 2 : -1;
                    }
                } else {
                    exhausted = true;
                }
            }
        }
        if (__ballot_sync(full, idx >= 0) == 0) break;

        // 2. one traversal round, while-while: an interior phase in which every
        //    lane descends until it stands at a leaf (or its stack runs out),
        //    then a leaf phase in which the lanes at a leaf test its triangles.
        bool fin = false;
        const bool live = idx >= 0;
        const bool shadow = (rfl & kRayShadow) != 0;
        for (int it = 0; it < kTraceSteps; ++it) {
            const bool act = live && !fin && node >= 0;
            if (!__any_sync(full, act)) break;
            if (act) {
                if (COUNT) ++tc.nodes;
                const float4 n0 = __ldg(g.nodes + 4 * node + 0), n1 = __ldg(g.nodes + 4 * node + 1),
                             n2 = __ldg(g.nodes + 4 * node + 2), n3 = __ldg(g.nodes + 4 * node + 3);
                float ta, tb;
                bool ha, hb;
                child_boxes(ray, n0, n1, n2, tmin, tw, ta, tb, ha, hb);
                int ca = __float_as_int(n3.x), cb = __float_as_int(n3.y);
                if (CHECKED) {
                    if (ca >= g.node_cap) {
                        trace_check_fail(a.err, 9, node, ca);
                        ca = ~0;
                    }
                    if (cb >= g.node_cap) {
                        trace_check_fail(a.err, 9, node, cb);
                        cb = ~0;
                    }
                }
                if (ha && hb) {
                    const bool a_first = shadow || ta <= tb;
                    if (sp < kStackSize) {
                        stack[sp++] = a_first ? cb : ca;
                    } else {
                        atomicCAS(a.err, 0, 5);   // deeper than the builder allows
                    }
                    node = a_first ? ca : cb;
                } else if (ha) {
                    node = ca;
                } else if (hb) {
                    node = cb;
                } else if (sp == 0) {
                    fin = true;
                } else {
                    node = stack[--sp];
                }
            }
        }
        if (live && !fin && node < 0) {
            const int v = ~node;
            const int first = v >> kLeafBits;
            int count = v & ((1 << kLeafBits) - 1);
            if (CHECKED && (int64_t)first + count > g.tri_cap) {
                trace_check_fail(a.err, 10, first, count);
                count = 0;
            }
            for (int i = 0; i < count; ++i) {
                const float4 *tp = g.tris + 3 * (first + i);
                const float4 ta4 = __ldg(tp), tb4 = __ldg(tp + 1), tc4 = __ldg(tp + 2);
                const int id = __float_as_int(ta4.w);
                if (shadow) {
                    if (id == excl) continue;
                    if (COUNT) ++tc.tris;
                    const float t = wt_intersect(ray, xyz(ta4), xyz(tb4), xyz(tc4));
                    if (!(t > tmin && t <= tw)) continue;
                    if (!(__float_as_uint(tc4.w) & kTriGlass)) {
                        occ = true;
                        break;
                    }
                    if (dot(ray.d, cross(xyz(tb4) - xyz(ta4), xyz(tc4) - xyz(ta4))) >= 0.0f) continue;   // leaving face
                    const int ob = __float_as_int(tb4.w);
                    bool seen = false;
                    for (int k = 0; k < cr.n; ++k) seen |= cr.obj[k] == ob;
                    if (seen) continue;
                    if (cr.n >= kMaxCross) {
                        occ = true;
                        break;
                    }
                    cr.obj[cr.n] = ob;
                    cr.tri[cr.n] = id;
                    ++cr.n;
                } else {
                    if (id == ep || (eo >= 0 && __float_as_int(tb4.w) == eo)) continue;
                    if (COUNT) ++tc.tris;
                    const float t = wt_intersect(ray, xyz(ta4), xyz(tb4), xyz(tc4));
                    if (t > tmin && (t < tw || (t == tw && (best < 0 || id < best)))) {
                        tw = t;
                        best = id;
                    }
                }
            }
            if (occ || sp == 0) {
                fin = true;
            } else {
                node = stack[--sp];
            }
        }

        // 3. finished lanes: final result, or hand-off to the neighbouring cell
        bool want = false;
        float4 o0 = make_float4(0, 0, 0, 0), o1 = o0;
        int4 o2 = make_int4(0, 0, 0, 0);
        if (fin) {
            bool done = false;
            int rfl_next = rfl;
            if (rfl & kRayShadow) {
                for (int k = n_prev; k < cr.n; ++k) {
                    const float4 cn = __ldg(a.sc.tri_n + cr.tri[k]);
                    a.ps.cross_obj[k * np + q] = cr.obj[k];
                    a.ps.cross_mat[k * np + q] = __float_as_int(cn.w);
                    a.ps.cross_cos[k * np + q] = -dot(ray.d, xyz(cn));
                }
                if (occ) {
                    a.ps.sh_status[q] = kShadowOccluded;
                    done = true;
                } else if (t_exit + g.eps >= t_max || next < 0) {
                    a.ps.sh_status[q] = kShadowClear | (cr.n << 4);
                    done = true;
                }
                rfl_next = (rfl & 1) | (cr.n << 1);
            } else {
                if (best >= 0) {
                    const V3 x = ray.o + tw * ray.d;
                    a.ps.hit0[q] = make_float4(x.x, x.y, x.z, __int_as_float(best));
                    a.ps.hit1[q] = make_float4(ray.d.x, ray.d.y, ray.d.z, tw);
                    done = true;
                } else if (next < 0) {
                    a.ps.hit0[q] = make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
                    a.ps.hit1[q] = make_float4(ray.d.x, ray.d.y, ray.d.z, 0.f);
                    done = true;
                }
            }
            if (!done && a.g.continue_cells) {
                // the lane carries the ray on into the neighbouring cell's
                // BVH, with the same record it would have handed over
                const int cell = next;
                t_cur = fmaxf(t_cur, t_exit);
                t_exit = cell_exit(g, cell, ray, next);
                tmin = fmaxf(0.0f, t_cur - g.eps);
                node = __ldg(g.root + cell);
                sp = 0;
                best = -1;
                occ = false;
                rfl = rfl_next;
                n_prev = cr.n;
                tw = (rfl & kRayShadow) ? fminf(t_exit + g.eps, t_max) : t_exit + g.eps;
                ++n_cross;
                ++n_vis;
                if (COUNT) ++n_cont;
                done = true;
                fin = false;
            } else {
                if (!done) {
                    want = true;
                    o0 = make_float4(ray.o.x, ray.o.y, ray.o.z, fmaxf(t_cur, t_exit));
                    o1 = make_float4(ray.d.x, ray.d.y, ray.d.z, t_max);
                    o2 = make_int4(q, excl, rfl_next, next);
                    ++n_cross;
                }
                idx = -1;
            }
        }
        if (want && a.last_wave) {   // cannot happen: each wave moves a ray forward along one axis
            atomicCAS(a.err, 0, 4);
            want = false;
        }
        // hand-off: append to the warp's buffer, flushing it to the staging
        // area (one atomic, coalesced stores) when the new rays do not fit
        const unsigned mw = __ballot_sync(full, want);
        if (mw) {
            const int n = __popc(mw);
            if (nbuf + n > kPushBuf) {
                flush_push_buf(Q, pbuf, nbuf, lane, a.err);
                nbuf = 0;
            }
            if (want) {
                float4 *slot = pbuf + 3 * (nbuf + __popc(mw & lt_mask));
                slot[0] = o0;
                slot[1] = o1;
                slot[2] = make_float4(__int_as_float(o2.x), __int_as_float(o2.y), __int_as_float(o2.z),
                                      __int_as_float(o2.w));
                const int bin = ray_bin(g, next, o2.z, o0, o1);
                const unsigned peers = __match_any_sync(mw, bin);
                if (lane == __ffs(peers) - 1) atomicAdd(Q.cnt + bin, __popc(peers));
            }
            nbuf += n;
            __syncwarp();
        }
    }
    if (nbuf > 0) flush_push_buf(Q, pbuf, nbuf, lane, a.err);
    block_count3(a.counters + 3, n_cross, nullptr, 0, nullptr, 0);
    if (COUNT) {
        __syncthreads();
        block_count3(a.counters + 5, tc.nodes, a.counters + 6, tc.tris, a.counters + 7, n_vis);
        __syncthreads();   // the reduction's shared slots are read by thread 0 above
        block_count3(a.counters + 10, n_cont, nullptr, 0, nullptr, 0);
    }
}
