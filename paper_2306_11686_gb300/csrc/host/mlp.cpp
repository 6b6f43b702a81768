/*
 * Learned launch shapes: features and the FP32 MLP forward pass (host C++).
 *
 * The model maps (loop features, shape features) to a predicted log of the
 * loop's run time; the chosen shape is the argmin over the candidate set.
 * The autotuner (exhaustive measurement over the same set) is the fallback
 * and the yardstick of the model's regret.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "gf.h"

static float lg2(double v) { return (float)log2(v > 1e-30 ? v : 1e-30); }

extern "C" GF_API void gf_tune_features(const gf_synth_loop *L, const gf_shape *sh, uint32_t sms, float *out)
{
    out[0] = lg2((double)(L->trip > 0 ? L->trip : 1));
    out[1] = lg2((double)L->bytes);
    out[2] = lg2((double)(L->flops ? L->flops : 1));
    out[3] = (float)((double)L->div_thresh / 4294967296.0);
    out[4] = (float)(1000.0 * (double)L->rpc_thresh / 4294967296.0);
    out[5] = lg2((double)sh->grid / (double)(sms ? sms : 1));
    out[6] = lg2((double)sh->block);
    out[7] = lg2((double)sh->chunk);
    out[8] = (float)sh->sched;
}

extern "C" GF_API int gf_mlp_forward(const float *P, int nin, int width, int depth, const float *x, int n, float *y)
{
    if (!P || !x || !y || nin < 1 || width < 1 || depth < 1 || n < 0)
        return GF_EINVAL;
    const float *mean = P, *sd = P + nin;
    std::vector<float> a((size_t)(nin > width ? nin : width)), b((size_t)width);
    for (int r = 0; r < n; r++) {
        for (int k = 0; k < nin; k++)
            a[(size_t)k] = (x[(size_t)r * nin + k] - mean[k]) / sd[k];
        const float *w = P + 2 * nin;
        int in = nin;
        for (int l = 0; l < depth; l++) {
            const float *bias = w + (size_t)width * in;
            for (int o = 0; o < width; o++) {
                float s = bias[o];
                const float *row = w + (size_t)o * in;
                for (int k = 0; k < in; k++)
                    s += row[k] * a[(size_t)k];
                b[(size_t)o] = s > 0.0f ? s : 0.0f;
            }
            for (int o = 0; o < width; o++)
                a[(size_t)o] = b[(size_t)o];
            w = bias + width;
            in = width;
        }
        float s = w[width];
        for (int k = 0; k < width; k++)
            s += w[k] * a[(size_t)k];
        y[r] = s;
    }
    return GF_OK;
}

extern "C" GF_API int gf_mlp_topk(const float *P, int width, int depth, const gf_synth_loop *L,
                                  const gf_shape *shapes, int nshapes, uint32_t sms, int k, int *idx)
{
    if (!P || !L || !shapes || nshapes < 1 || !idx || k < 1 || k > nshapes)
        return GF_EINVAL;
    std::vector<float> f((size_t)nshapes * GF_TUNE_NFEAT), y((size_t)nshapes);
    for (int s = 0; s < nshapes; s++)
        gf_tune_features(L, &shapes[s], sms, &f[(size_t)s * GF_TUNE_NFEAT]);
    int rc = gf_mlp_forward(P, GF_TUNE_NFEAT, width, depth, f.data(), nshapes, y.data());
    if (rc)
        return rc;
    std::vector<int> order((size_t)nshapes);
    for (int s = 0; s < nshapes; s++)
        order[(size_t)s] = s;
    std::partial_sort(order.begin(), order.begin() + k, order.end(),
                      [&](int a, int b) { return y[(size_t)a] < y[(size_t)b] || (y[(size_t)a] == y[(size_t)b] && a < b); });
    for (int j = 0; j < k; j++)
        idx[j] = order[(size_t)j];
    return GF_OK;
}

extern "C" GF_API int gf_mlp_choose(const float *P, int width, int depth, const gf_synth_loop *L,
                                    const gf_shape *shapes, int nshapes, uint32_t sms, int *best)
{
    return gf_mlp_topk(P, width, depth, L, shapes, nshapes, sms, 1, best);
}
