// Les Houches Event file writer (LHE 3.0 text), running in its own thread so
// that formatting and file output overlap the integration (Sec. 2.5: the
// unweighted events are written asynchronously by a separate writer).
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "mf_internal.h"

using mfi::fail;

struct mf_lhe_writer {
    std::FILE *f = nullptr;
    mf_lhe_init init{};
    std::thread th;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<std::vector<double>> q;      // batches of records [n][4 + 4 n_legs]
    std::vector<int32_t> tags;              // [n_flows][n_legs][2] colour, anticolour
    bool closing = false;
    bool io_error = false;
    int64_t written = 0;
};

namespace {

// One event: weight, then per leg PDG id, status, mothers, colour and
// anticolour tags of the event's colour flow (0 where the flow index is
// outside the table), momentum (px, py, pz, E), mass, lifetime, spin
// (unknown).
void write_event(mf_lhe_writer *w, const double *rec) {
    const mf_lhe_init &in = w->init;
    const int n = in.n_legs;
    std::FILE *f = w->f;
    const int flow = (int)rec[3];
    const int32_t *tag = (flow >= 0 && flow < in.n_flows && !w->tags.empty())
                             ? w->tags.data() + (size_t)flow * n * 2 : nullptr;
    std::fprintf(f, "<event>\n%d %d %.10e %.8e %.8e %.8e\n", n, in.process_id, rec[0], in.scale, in.alpha_qed,
                 in.alpha_s);
    for (int i = 0; i < n; ++i) {
        const double *p = rec + 4 + 4 * i;
        const int incoming = i < 2;
        const double m = in.mass[i];
        std::fprintf(f, " %8d %2d %4d %4d %4d %4d %+.12e %+.12e %+.12e %.12e %.8e %.1f %.1f\n", in.pdg[i],
                     incoming ? -1 : 1, incoming ? 0 : 1, incoming ? 0 : 2, tag ? tag[2 * i] : 0,
                     tag ? tag[2 * i + 1] : 0, p[1], p[2], p[3], p[0], m, 0.0, 9.0);
    }
    std::fprintf(f, "</event>\n");
}

void run(mf_lhe_writer *w) {
    const int rec = 4 + 4 * w->init.n_legs;
    for (;;) {
        std::vector<double> batch;
        {
            std::unique_lock<std::mutex> lock(w->mu);
            w->cv.wait(lock, [&] { return w->closing || !w->q.empty(); });
            if (w->q.empty()) return;                 // closing and drained
            batch = std::move(w->q.front());
            w->q.pop_front();
        }
        const size_t n = batch.size() / rec;
        for (size_t k = 0; k < n; ++k) write_event(w, batch.data() + k * rec);
        bool bad = std::ferror(w->f) != 0;
        std::lock_guard<std::mutex> lock(w->mu);
        w->written += (int64_t)n;
        w->io_error |= bad;
        w->cv.notify_all();
    }
}

}  // namespace

namespace mfi {
// Hand a batch of records (4 + 4 n_legs doubles each) to the writer thread.
mf_status lhe_push(mf_lhe_writer *w, std::vector<double> &&records) {
    if (records.empty()) return MF_OK;
    std::lock_guard<std::mutex> lock(w->mu);
    if (w->closing) return fail(MF_EINVAL, "LHE writer is closed");
    w->q.push_back(std::move(records));
    w->cv.notify_all();
    return MF_OK;
}
int lhe_legs(const mf_lhe_writer *w) { return w->init.n_legs; }
}  // namespace mfi

extern "C" mf_status mf_lhe_open(const char *path, const mf_lhe_init *init, mf_lhe_writer **out) {
    if (!out) return fail(MF_EINVAL, "out is NULL");
    *out = nullptr;
    if (!path || !init) return fail(MF_EINVAL, "NULL argument");
    if (init->n_legs < 3 || init->n_legs > MF_MAX_LEGS) return fail(MF_EINVAL, "n_legs out of range");
    if (init->n_flows < 0 || (init->n_flows > 0 && !init->colour_tags)) return fail(MF_EINVAL, "bad colour tags");
    std::FILE *f = std::fopen(path, "w");
    if (!f) return fail(MF_EINVAL, std::string("cannot open ") + path);
    mf_lhe_writer *w = new (std::nothrow) mf_lhe_writer();
    if (!w) {
        std::fclose(f);
        return fail(MF_ENOMEM, "host allocation");
    }
    w->f = f;
    w->init = *init;
    if (init->n_flows > 0)
        w->tags.assign(init->colour_tags, init->colour_tags + (size_t)init->n_flows * init->n_legs * 2);
    w->init.colour_tags = nullptr;            // the copy above is used
    // header and the <init> block: beams, PDF sets (none: -1), weighting
    // strategy 3 (unweighted), one process with its cross section
    std::fprintf(f, "<LesHouchesEvents version=\"3.0\">\n<header>\n<generator name=\"madflow-gb300\" />\n</header>\n");
    std::fprintf(f, "<init>\n%d %d %.8e %.8e %d %d %d %d %d %d\n", init->beam_pdg[0], init->beam_pdg[1],
                 init->beam_energy[0], init->beam_energy[1], -1, -1, -1, -1, 3, 1);
    std::fprintf(f, "%.10e %.10e %.10e %d\n</init>\n", init->xsec, init->xsec_error, init->w_max, init->process_id);
    w->th = std::thread(run, w);
    *out = w;
    return MF_OK;
}

extern "C" mf_status mf_lhe_write(mf_lhe_writer *w, const double *records, int64_t n) {
    if (!w || (n > 0 && !records) || n < 0) return fail(MF_EINVAL, "bad arguments");
    const size_t rec = 4 + 4 * (size_t)w->init.n_legs;
    return mfi::lhe_push(w, std::vector<double>(records, records + rec * (size_t)n));
}

extern "C" mf_status mf_lhe_close(mf_lhe_writer *w, int64_t *n_written) {
    if (!w) return MF_OK;
    {
        std::lock_guard<std::mutex> lock(w->mu);
        w->closing = true;
        w->cv.notify_all();
    }
    if (w->th.joinable()) w->th.join();
    std::fprintf(w->f, "</LesHouchesEvents>\n");
    const bool bad = w->io_error || std::ferror(w->f) != 0;
    const bool close_bad = std::fclose(w->f) != 0;
    if (n_written) *n_written = w->written;
    delete w;
    if (bad || close_bad) return fail(MF_EINVAL, "LHE file write failed");
    return MF_OK;
}
