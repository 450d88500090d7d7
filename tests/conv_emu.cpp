// Test driver: one convolution layer of the learned-guess network through the
// library's own tensor-core kernels (forward, input gradient, weight and bias
// gradients, weight repacking), compiled for the host with the shim of
// host_kernel_shim.h.  The kernels come from cnn.cu (conv_kernels.inc, written
// by the test); BF16 is emulated here with round-to-nearest-even, and
// mma.sync.m16n8k16 (BF16 in, FP32 accumulate) and ldmatrix.x4 by exchanges
// between the lanes of a warp, in the register layouts the PTX ISA documents
// (the mma's, below; ldmatrix's, at emu_ldsm):
//   A (16 x 16, row): lane 4 (r % 8) + (k % 8) / 2, register (r >= 8) + 2 (k >= 8), half k % 2
//   B (16 x 8, col):  lane 4 n + (k % 8) / 2,       register (k >= 8),             half k % 2
//   C (16 x 8):       lane 4 (r % 8) + n / 2,       register 2 (r >= 8) + n % 2
// The test's values are small integers (and multiples of 2^-8), so every sum
// is exact in any order and the results are compared exactly.
//
// usage: conv_emu DIR B Hin Win ksz stride ca cb cout
// reads DIR/{in_a,in_b,gout,act_a,act_b}.bf16 (uint16 bits), DIR/{w,bias,add_a}.f32;
// writes DIR/{fwd.bf16, fwd_nchw.f32, gin_a.bf16, gin_b.f32, gw.f32, gb.f32}
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

#include "host_kernel_shim.h"

#define __align__(n) __attribute__((aligned(n)))

struct __nv_bfloat16 {
    uint16_t x;
};
inline __nv_bfloat16 __float2bfloat16(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    const uint32_t r = (u + 0x7FFFu + ((u >> 16) & 1u)) >> 16;
    return __nv_bfloat16{(uint16_t)r};
}
inline float __bfloat162float(__nv_bfloat16 h) {
    const uint32_t u = (uint32_t)h.x << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}
struct alignas(16) uint4 {
    uint32_t x, y, z, w;
};
inline uint4 make_uint4(uint32_t a, uint32_t b, uint32_t c, uint32_t d) { return uint4{a, b, c, d}; }

inline std::vector<uint32_t>* emu_frag = nullptr;  // 6 words per thread: a[4], b[2]

inline float emu_half(uint32_t w, int h) { return __bfloat162float(__nv_bfloat16{(uint16_t)(h ? w >> 16 : w & 0xFFFFu)}); }

inline void mma_bf16_16816(float* c, const uint32_t* a, const uint32_t* b) {
    const int t = threadIdx.x, w = t >> 5, lane = t & 31;
    for (int i = 0; i < 4; ++i) (*emu_frag)[t * 6 + i] = a[i];
    for (int i = 0; i < 2; ++i) (*emu_frag)[t * 6 + 4 + i] = b[i];
    __syncwarp();
    auto A = [&](int r, int k) {
        const int l = 4 * (r % 8) + (k % 8) / 2, reg = (r >= 8 ? 1 : 0) + (k >= 8 ? 2 : 0);
        return emu_half((*emu_frag)[(w * 32 + l) * 6 + reg], k % 2);
    };
    auto B = [&](int k, int n) {
        const int l = 4 * n + (k % 8) / 2, reg = k >= 8 ? 1 : 0;
        return emu_half((*emu_frag)[(w * 32 + l) * 6 + 4 + reg], k % 2);
    };
    float out[4];
    for (int e = 0; e < 4; ++e) {
        const int r = lane / 4 + 8 * (e >> 1), n = 2 * (lane % 4) + (e & 1);
        double s = 0.0;
        for (int k = 0; k < 16; ++k) s += (double)A(r, k) * (double)B(k, n);
        out[e] = (float)((double)c[e] + s);
    }
    __syncwarp();
    for (int e = 0; e < 4; ++e) c[e] = out[e];
}

// ldmatrix.x4 (and .trans): lane l names row l % 8 of matrix l / 8; register j of
// lane t gets row t / 4, columns 2 (t % 4), 2 (t % 4) + 1 of matrix j (low half
// first), or with .trans rows 2 (t % 4), 2 (t % 4) + 1 of column t / 4
inline std::vector<const void*>* emu_rows = nullptr;

inline void emu_ldsm(uint32_t* r, const __nv_bfloat16* p, bool trans) {
    const int t = threadIdx.x, w = t >> 5, lane = t & 31;
    (*emu_rows)[t] = p;
    __syncwarp();
    for (int j = 0; j < 4; ++j) {
        uint16_t h[2];
        for (int e = 0; e < 2; ++e) {
            const int row = trans ? 2 * (lane % 4) + e : lane / 4, col = trans ? lane / 4 : 2 * (lane % 4) + e;
            h[e] = static_cast<const __nv_bfloat16*>((*emu_rows)[w * 32 + 8 * j + row])[col].x;
        }
        r[j] = (uint32_t)h[0] | ((uint32_t)h[1] << 16);
    }
    __syncwarp();
}
inline void ldsm_x4(uint32_t* r, const __nv_bfloat16* p) { emu_ldsm(r, p, false); }
inline void ldsm_x4_trans(uint32_t* r, const __nv_bfloat16* p) { emu_ldsm(r, p, true); }

// cp.async: the copy (or the zero fill) happens at once, so commit and wait have nothing to do; the
// pipeline's group accounting is checked on the GPU, its addresses and predicates here
inline void cp_async16(__nv_bfloat16* dst, const __nv_bfloat16* src, bool valid) {
    if (valid) std::memcpy(dst, src, 16);
    else std::memset(dst, 0, 16);
}
inline void cp_async_commit() {}
template <int N>
inline void cp_async_wait() {}

#include "conv_kernels.inc"

template <class T>
std::vector<T> load(const std::string& path, size_t n) {
    std::vector<T> v(n);
    FILE* f = std::fopen(path.c_str(), "rb");
    if (!f || std::fread(v.data(), sizeof(T), n, f) != n) {
        std::fprintf(stderr, "cannot read %s\n", path.c_str());
        std::exit(2);
    }
    std::fclose(f);
    return v;
}
template <class T>
void save(const std::string& path, const std::vector<T>& v) {
    FILE* f = std::fopen(path.c_str(), "wb");
    std::fwrite(v.data(), sizeof(T), v.size(), f);
    std::fclose(f);
}

// every block of a grid (x, y, z) of kGemmThreads threads
template <class F>
void launch3(int gx, int gy, int gz, int threads, F body) {
    std::vector<uint32_t> frag((size_t)threads * 6, 0u);
    std::vector<const void*> rows((size_t)threads, nullptr);
    emu_frag = &frag;
    emu_rows = &rows;
    for (int z = 0; z < gz; ++z)
        for (int y = 0; y < gy; ++y) {
            blockIdx.y = y;
            blockIdx.z = z;
            gridDim.y = gy;
            gridDim.z = gz;
            emu_launch(gx, threads, 0, body);
        }
}

int main(int argc, char** argv) {
    if (argc != 10) return 1;
    const std::string d = argv[1];
    const int B = std::atoi(argv[2]), Hin = std::atoi(argv[3]), Win = std::atoi(argv[4]), ksz = std::atoi(argv[5]),
              stride = std::atoi(argv[6]), ca = std::atoi(argv[7]), cb = std::atoi(argv[8]), cout = std::atoi(argv[9]);
    auto p16 = [](int c) { return (c + 15) / 16 * 16; };
    ConvGeom g;
    g.B = B; g.Hin = Hin; g.Win = Win; g.Hout = (Hin + stride - 1) / stride; g.Wout = (Win + stride - 1) / stride;
    g.ksz = ksz; g.stride = stride; g.pad = ksz / 2; g.taps = ksz * ksz;
    g.ca = ca; g.Ka = p16(ca); g.cb = cb; g.Kb = cb ? p16(cb) : 0; g.Kc = g.Ka + g.Kb; g.cout = cout; g.Np = p16(cout);
    const size_t pin = (size_t)B * Hin * Win, pout = (size_t)B * g.Hout * g.Wout, cin = ca + cb;
    auto in_a = load<__nv_bfloat16>(d + "/in_a.bf16", pin * g.Ka);
    auto in_b = cb ? load<__nv_bfloat16>(d + "/in_b.bf16", pin * g.Kb) : std::vector<__nv_bfloat16>(1);
    auto act_a = load<__nv_bfloat16>(d + "/act_a.bf16", pin * g.Ka);
    auto act_b = cb ? load<__nv_bfloat16>(d + "/act_b.bf16", pin * g.Kb) : std::vector<__nv_bfloat16>(1);
    auto add_a = load<float>(d + "/add_a.f32", pin * g.Ka);
    auto gout = load<__nv_bfloat16>(d + "/gout.bf16", pout * g.Np);
    auto w = load<float>(d + "/w.f32", (size_t)cout * cin * g.taps);
    auto bias = load<float>(d + "/bias.f32", cout);

    std::vector<__nv_bfloat16> wf((size_t)g.Np * g.taps * g.Kc), wb(wf.size());
    emu_launch((int)((wf.size() + 255) / 256), 256, 0, [&] { repack_kernel(g, w.data(), wf.data(), wb.data()); });

    // forward with ReLU to BF16, and without ReLU to FP32 [b][cout][y][x]
    std::vector<__nv_bfloat16> fwd(pout * g.Np);
    std::vector<float> fwd_nchw(pout * cout);
    {
        GemmArgs a;
        std::memset(&a, 0, sizeof(a));
        a.g = g;
        a.M = (int)pout; a.N = g.Np; a.K = g.taps * g.Kc;
        a.in_a = in_a.data(); a.in_b = cb ? in_b.data() : nullptr; a.wt = wf.data(); a.bias = bias.data();
        a.wt_ld = a.K;
        a.relu = 1; a.out_bf = fwd.data();
        launch3((a.M + kBM - 1) / kBM, (a.N + kBN - 1) / kBN, 1, kGemmThreads, [&] { conv_gemm_kernel<kFwd>(a); });
        a.relu = 0; a.out_bf = nullptr; a.out_nchw = fwd_nchw.data();
        launch3((a.M + kBM - 1) / kBM, (a.N + kBN - 1) / kBN, 1, kGemmThreads, [&] { conv_gemm_kernel<kFwd>(a); });
    }
    // input gradient: part a masked, plus add_a, to BF16; part b masked, to FP32
    std::vector<__nv_bfloat16> gin_a(pin * g.Ka);
    std::vector<float> gin_b(cb ? pin * g.Kb : 1);
    {
        GemmArgs a;
        std::memset(&a, 0, sizeof(a));
        a.g = g;
        a.M = (int)pin; a.N = g.Kc; a.K = g.taps * g.Np;
        a.gout = gout.data(); a.wt = wb.data(); a.wt_ld = a.K;
        a.part[0] = GradPart{act_a.data(), add_a.data(), gin_a.data(), nullptr, g.Ka};
        if (cb) a.part[1] = GradPart{act_b.data(), nullptr, nullptr, gin_b.data(), g.Kb};
        if (stride == 1) {
            launch3((a.M + kBM - 1) / kBM, (a.N + kBN - 1) / kBN, 1, kGemmThreads,
                    [&] { conv_gemm_kernel<kBwdData>(a); });
        } else {
            // as the library launches a strided layer's input gradient: one launch per parity class
            a.cls = 1;
            a.M = B * (Hin / stride) * (Win / stride);
            for (int py = 0; py < stride; ++py)
                for (int px = 0; px < stride; ++px) {
                    a.py = py;
                    a.px = px;
                    a.ntap = class_taps(g, py, px, a.tapk);
                    a.K = a.ntap * g.Np;
                    std::printf("class (%d, %d): %d taps\n", py, px, a.ntap);
                    launch3((a.M + kBM - 1) / kBM, (a.N + kBN - 1) / kBN, 1, kGemmThreads,
                            [&] { conv_gemm_kernel<kBwdData>(a); });
                }
        }
    }
    // weight and bias gradients through the split partials
    std::vector<float> gw((size_t)cout * cin * g.taps), gb(cout);
    {
        GemmArgs a;
        std::memset(&a, 0, sizeof(a));
        a.g = g;
        a.M = g.Np; a.N = g.taps * g.Kc; a.K = (int)pout;
        a.in_a = in_a.data(); a.in_b = cb ? in_b.data() : nullptr; a.gout = gout.data();
        const long long tiles = (long long)((a.M + kBM - 1) / kBM) * ((a.N + kBN - 1) / kBN);
        int splits = 1;
        weight_splits(a.K, tiles, &splits, &a.kchunk);
        std::vector<float> wpart((size_t)splits * g.Np * a.N, -1.0f);
        a.wpart = wpart.data();
        launch3((a.M + kBM - 1) / kBM, (a.N + kBN - 1) / kBN, splits, kGemmThreads,
                [&] { conv_gemm_kernel<kBwdWeight>(a); });
        const int chunk = std::atoi(std::getenv("BIAS_CHUNK") ? std::getenv("BIAS_CHUNK") : "1024");
        const int bsplits = (a.K + chunk - 1) / chunk;
        std::vector<float> bpart((size_t)bsplits * g.Np, -1.0f);
        launch3((g.Np + 63) / 64, bsplits, 1, 256, [&] { bias_partial_kernel(a.K, g.Np, chunk, gout.data(), bpart.data()); });
        const long long nw = (long long)cout * cin * g.taps;
        emu_launch((int)((nw + cout + 255) / 256), 256, 0,
                   [&] { grad_reduce_kernel(g, splits, wpart.data(), bsplits, bpart.data(), gw.data(), gb.data()); });
        std::printf("splits %d kchunk %d bias splits %d\n", splits, a.kchunk, bsplits);
    }
    save(d + "/fwd.bf16", fwd);
    save(d + "/fwd_nchw.f32", fwd_nchw);
    save(d + "/gin_a.bf16", gin_a);
    if (cb) save(d + "/gin_b.f32", gin_b);
    save(d + "/gw.f32", gw);
    save(d + "/gb.f32", gb);
    return 0;
}
