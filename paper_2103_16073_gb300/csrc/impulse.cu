// Broadband responses (Sec. 4, Eqs. an1-an3): the image-source field of a
// shoebox room at many frequencies (the analytical comparison of Sec. 4) and
// the time-domain synthesis of a pulse response from frequency-domain
// solutions at equispaced frequencies.
#include <cmath>
#include <vector>

#include "common.cuh"

namespace {

constexpr double kPi = 3.14159265358979323846;

// out[m * nr + r] = sum_j A_j e^{i k_m R_j} / (4 pi R_j), R_j = |rcv_r - img_j|
__global__ void k_image_field(const double* __restrict__ img, const cd* __restrict__ amp, int64_t nimg,
                              const double* __restrict__ kk, int nf, const double* __restrict__ rcv, int64_t nr,
                              cd* __restrict__ out) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nr * nf) return;
    int64_t r = t % nr;
    int m = (int)(t / nr);
    double k = kk[m];
    double x = rcv[3 * r], y = rcv[3 * r + 1], z = rcv[3 * r + 2];
    cd acc = mk(0.0, 0.0);
    for (int64_t j = 0; j < nimg; ++j) {
        double dx = x - img[3 * j], dy = y - img[3 * j + 1], dz = z - img[3 * j + 2];
        double R = sqrt(dx * dx + dy * dy + dz * dz);
        double s, c;
        sincos(k * R, &s, &c);
        double w = 1.0 / (4.0 * kPi * R);
        acc = acc + amp[j] * mk(c * w, s * w);
    }
    out[t] = acc;
}

// out[n * nr + r] = 2 df Re sum_m psi[m * nr + r] F_m e^{-i 2 pi f_m t_n},
// F_m = 2 i sin(2 pi f_m Dt) (the pulse of Eq. an3), t_n = n dt
__global__ void k_pulse_synth(const cd* __restrict__ psi, const double* __restrict__ f, int nf, int64_t nr,
                              double df, double dt, int nt, double pulse_dt, double* __restrict__ out) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nr * (int64_t)nt) return;
    int64_t r = t % nr;
    int n = (int)(t / nr);
    double tn = n * dt;
    double acc = 0.0;
    for (int m = 0; m < nf; ++m) {
        double w = 2.0 * kPi * f[m];
        double s, c;
        sincos(-w * tn, &s, &c);
        double F = 2.0 * sin(w * pulse_dt);   // F = i F
        cd P = psi[(int64_t)m * nr + r] * mk(0.0, F);
        acc += P.re * c - P.im * s;
    }
    out[t] = 2.0 * df * acc;
}

}  // namespace

// Image sources of Allen and Berkley for the room [0,lx]x[0,ly]x[0,lz]: per
// axis the coordinate 2 q L + (1 - 2u) s with |q - u| reflections off the
// wall at 0 and |q| off the wall at L; the amplitude is the product of the
// wall reflection coefficients over the reflections; images with |A| below
// a_th are dropped (the direct source is always kept).
fb_status fb_image_field_impl(const double* room, const double* src, const cd* Rw, double a_th, const double* k,
                              int nf, const double* rcv, int64_t nr, cd* out, cudaStream_t s) {
    double rmax = 0.0;
    for (int w = 0; w < 6; ++w) rmax = std::max(rmax, std::hypot(Rw[w].re, Rw[w].im));
    // images per axis: enough for |A| >= a_th, at most 2 x 64 + 2 (about
    // 2.2 million candidates in all); |R| >= 1 keeps 20 orders per axis
    const double qneed = rmax < 1.0 ? std::ceil(std::log(a_th) / std::log(rmax) / 2.0) + 1.0 : 20.0;
    if (!(qneed <= 64.0))
        return fb_fail(FB_ERR_ARG, "reflection coefficients this close to 1 need more than 64 image orders per "
                                   "axis for a_th; raise a_th");
    const int qmax = (int)qneed;
    struct Ax {
        std::vector<double> pos;
        std::vector<cd> amp;
        std::vector<int> nref;
    } ax[3];
    for (int d = 0; d < 3; ++d) {
        cd r0 = Rw[2 * d], r1 = Rw[2 * d + 1];
        for (int q = -qmax; q <= qmax; ++q)
            for (int u = 0; u < 2; ++u) {
                int n0 = std::abs(q - u), n1 = std::abs(q);
                cd a = mk(1.0, 0.0);
                for (int i = 0; i < n0; ++i) a = a * r0;
                for (int i = 0; i < n1; ++i) a = a * r1;
                ax[d].pos.push_back(2.0 * q * room[d] + (1 - 2 * u) * src[d]);
                ax[d].amp.push_back(a);
                ax[d].nref.push_back(n0 + n1);
            }
    }
    std::vector<double> img;
    std::vector<cd> amp;
    for (size_t i = 0; i < ax[0].pos.size(); ++i)
        for (size_t j = 0; j < ax[1].pos.size(); ++j)
            for (size_t l = 0; l < ax[2].pos.size(); ++l) {
                cd a = ax[0].amp[i] * ax[1].amp[j] * ax[2].amp[l];
                bool direct = ax[0].nref[i] + ax[1].nref[j] + ax[2].nref[l] == 0;
                if (!direct && std::hypot(a.re, a.im) < a_th) continue;
                img.push_back(ax[0].pos[i]);
                img.push_back(ax[1].pos[j]);
                img.push_back(ax[2].pos[l]);
                amp.push_back(a);
            }
    const int64_t nimg = (int64_t)amp.size();
    double *dimg = nullptr, *dk = nullptr;
    cd* damp = nullptr;
    auto done = [&](fb_status st) { dfree(dimg); dfree(dk); dfree(damp); return st; };
    fb_status st;
    if ((st = dalloc(&dimg, img.size())) || (st = dalloc(&damp, amp.size())) || (st = dalloc(&dk, (size_t)nf)))
        return done(st);
    cudaMemcpyAsync(dimg, img.data(), sizeof(double) * img.size(), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(damp, amp.data(), sizeof(cd) * amp.size(), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(dk, k, sizeof(double) * nf, cudaMemcpyHostToDevice, s);
    k_image_field<<<div_up(nr * nf, 128), 128, 0, s>>>(dimg, damp, nimg, dk, nf, rcv, nr, out);
    fb_count_launch();
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return done(fb_fail(FB_ERR_CUDA, std::string("image field: ") + cudaGetErrorString(e)));
    return done(FB_OK);
}

fb_status fb_pulse_synthesis_impl(const cd* psi, const double* freqs, int nf, int64_t nr, double df, double dt,
                                  int nt, double pulse_dt, double* out, cudaStream_t s) {
    double* dfq = nullptr;
    FB_CHECK(dalloc(&dfq, (size_t)nf));
    cudaMemcpyAsync(dfq, freqs, sizeof(double) * nf, cudaMemcpyHostToDevice, s);
    k_pulse_synth<<<div_up(nr * (int64_t)nt, 128), 128, 0, s>>>(psi, dfq, nf, nr, df, dt, nt, pulse_dt, out);
    fb_count_launch();
    cudaError_t e = cudaStreamSynchronize(s);
    dfree(dfq);
    if (e != cudaSuccess) return fb_fail(FB_ERR_CUDA, std::string("pulse synthesis: ") + cudaGetErrorString(e));
    return FB_OK;
}
