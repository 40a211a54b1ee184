/*
 * cluster.c - oracle of the event clustering of monolithic-scintillator
 * detections (Sec. 2 of the paper).
 *
 * TEST INFRASTRUCTURE ONLY (same rules as oracle.c: loaded by the tests, the
 * smoke check and the benchmark's CPU leg; shares nothing with the CUDA
 * library).
 *
 * Inputs: N detections sorted by time, integer time stamps t[i] (ticks) and
 * integer amplitudes adc[i] (ADC channels).  All arithmetic is integer, so
 * the GPU must agree bit for bit.
 *
 * Max-step clustering (Sec. 2, the three enumerated steps):
 *   1. the step between consecutive detections, dt = t[i+1] - t[i];
 *   2. the mask M_i = (dt < dt_max) on that step;
 *   3. the edge of detection i, E_i = M_{i-1} XOR M_i.
 * Reading: the first and the last detection have no step on their outer
 * side, taken as a mask of false; an isolated detection (no step below
 * dt_max on either side) therefore gets no edge and belongs to no event.
 * Steps are computed in two's-complement 64-bit arithmetic (wrapping), the
 * same expression on both sides; they are meaningful for |dt| < 2^63.
 *
 * Events from the edges: in time order the edges alternate between the
 * first and the last detection of an event (a run of detections joined by
 * masked steps); events are numbered 0, 1, ... in time order.
 *
 * Fixed-window clustering (the prior art that Sec. 2 replaces): a window of
 * length W opens at detection i; if the detections with t < t[i] + W number
 * at least n_min and their amplitudes sum to at least adc_min they form an
 * event and the next window opens at the first detection after them,
 * otherwise the window moves on by one detection.  Sequential by
 * construction; kept here only for comparisons.
 */
#include <stdint.h>

#include "oracle.h"

static int64_t step_of(int64_t a, int64_t b) {      /* b - a, wrapping */
    return (int64_t)((uint64_t)b - (uint64_t)a);
}

void or_maxstep_edges(const int64_t *t, int64_t N, int64_t dt_max, uint8_t *edge) {
    for (int64_t i = 0; i < N; i++) {
        int m_before = i > 0 ? step_of(t[i - 1], t[i]) < dt_max : 0;
        int m_after = i + 1 < N ? step_of(t[i], t[i + 1]) < dt_max : 0;
        edge[i] = (uint8_t)(m_before ^ m_after);
    }
}

int64_t or_events_from_edges(const uint8_t *edge, const uint32_t *adc, int64_t N,
                             int32_t *event_id, int64_t *first, int32_t *count,
                             uint64_t *adc_sum) {
    int64_t k = 0, begin = 0;
    int inside = 0;
    uint64_t s = 0;
    for (int64_t i = 0; i < N; i++) {
        if (!inside) {
            if (edge[i]) {               /* first detection of event k */
                inside = 1;
                begin = i;
                s = adc[i];
                event_id[i] = (int32_t)k;
            } else {
                event_id[i] = -1;        /* isolated */
            }
        } else {
            s += adc[i];
            event_id[i] = (int32_t)k;
            if (edge[i]) {               /* last detection of event k */
                first[k] = begin;
                count[k] = (int32_t)(i - begin + 1);
                adc_sum[k] = s;
                k++;
                inside = 0;
            }
        }
    }
    return k;
}

int64_t or_fixed_window(const int64_t *t, const uint32_t *adc, int64_t N, int64_t window,
                        int64_t n_min, uint64_t adc_min, int32_t *event_id, int64_t *first,
                        int32_t *count, uint64_t *adc_sum) {
    int64_t k = 0, i = 0;
    for (int64_t j = 0; j < N; j++) event_id[j] = -1;
    while (i < N) {
        int64_t j = i;
        uint64_t s = 0;
        while (j < N && step_of(t[i], t[j]) < window) s += adc[j++];
        if (j - i >= n_min && s >= adc_min) {
            for (int64_t m = i; m < j; m++) event_id[m] = (int32_t)k;
            first[k] = i;
            count[k] = (int32_t)(j - i);
            adc_sum[k] = s;
            k++;
            i = j;
        } else {
            i++;
        }
    }
    return k;
}

void or_spectrum(const uint64_t *adc_sum, int64_t K, uint64_t bin_width, int32_t nbins,
                 uint64_t *hist) {
    for (int32_t b = 0; b < nbins; b++) hist[b] = 0;
    for (int64_t k = 0; k < K; k++) {
        uint64_t b = adc_sum[k] / bin_width;
        hist[b < (uint64_t)nbins ? b : (uint64_t)nbins - 1]++;
    }
}
