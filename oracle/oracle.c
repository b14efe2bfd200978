/*
 * Oracle for "Simultaneous Finite Automata: An Efficient Data-Parallel Model
 * for Regular Expression Matching" (Sin'ya, Matsuzaki, Sassa, ICPP 2013).
 *
 * TEST INFRASTRUCTURE ONLY.  Plain, slow, obviously correct CPU code used by
 * the tests, by __graft_entry__.smoke() and by the CPU-baseline leg of
 * bench.py.  The CUDA product path never links, loads or calls it, and it
 * shares no code, header, table or constant with that path.
 *
 * Conventions: a DFA is a total table delta[q*256 + b] over the 256 byte
 * values (int32), an initial state and an accept vector (0/1 per state).
 * An SFA built here is numbered in discovery order: id 0 is the identity
 * mapping f_I, map[id*nq + q] = f(q), sfa_delta[id*nsym + k] = id of
 * f . delta^{symbols[k]} (the reverse composition of Sect. II-A).
 *
 * Pins: see the header of oracle/__init__.py; every function below is
 * pinned there (parity pinned).
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------
 * Alg. 2 (sequential computation of a DFA), extended with the number of
 * positions i in 1..n whose prefix w[1..i] leads to a final state.
 * Returns the final state; *count receives that number.
 * ---------------------------------------------------------------------- */
int32_t oracle_dfa_run(const int32_t *delta, int32_t nq, int32_t q_start,
                       const uint8_t *accept, const uint8_t *text, uint64_t n,
                       uint64_t *count)
{
    (void)nq;
    int32_t q = q_start;
    uint64_t c = 0;
    for (uint64_t i = 0; i < n; ++i) {
        q = delta[(int64_t)q * 256 + text[i]];
        c += accept[q] ? 1u : 0u;
    }
    if (count) *count = c;
    return q;
}

/* ------------------------------------------------------------------------
 * Alg. 4 (correspondence construction) for a DFA, with the simplification
 * of Sect. V-A: f_next(q) = delta(q', sigma) where {q'} = f(q).
 * Q_tmp is a FIFO queue (the paper leaves the choice open); symbols are
 * taken in the order given.  Membership "f_next not in Q_s" is decided by
 * an open-addressing hash set over the mapping vectors.
 *
 * out_map      [cap * nq]   mapping of every SFA state
 * out_delta    [cap * nsym] SFA transition table (ids)
 * out_parent   [cap]        BFS parent id (-1 for f_I)
 * out_psym     [cap]        index of the symbol on the edge from the parent
 * Returns |Q_s|, or -1 when more than cap states are reached.
 * ---------------------------------------------------------------------- */
static uint64_t hash_vec(const int32_t *v, int32_t nq)
{
    uint64_t h = 1469598103934665603ull;           /* FNV-1a, 64 bit */
    for (int32_t i = 0; i < nq; ++i) {
        uint32_t x = (uint32_t)v[i];
        for (int k = 0; k < 4; ++k) {
            h ^= (x >> (8 * k)) & 0xffu;
            h *= 1099511628211ull;
        }
    }
    return h;
}

int64_t oracle_sfa_build(const int32_t *delta, int32_t nq, const uint8_t *symbols,
                         int32_t nsym, int64_t cap, int32_t *out_map,
                         int32_t *out_delta, int32_t *out_parent, int32_t *out_psym)
{
    if (cap < 1 || nq < 1) return -1;
    uint64_t hsize = 1;
    while (hsize < (uint64_t)cap * 2) hsize <<= 1;
    int64_t *slot = (int64_t *)malloc(hsize * sizeof(int64_t));
    int32_t *fnext = (int32_t *)malloc((size_t)nq * sizeof(int32_t));
    if (!slot || !fnext) { free(slot); free(fnext); return -2; }
    for (uint64_t i = 0; i < hsize; ++i) slot[i] = -1;

    /* Q_tmp <- {f_I} */
    int64_t count = 1;
    for (int32_t q = 0; q < nq; ++q) out_map[q] = q;
    out_parent[0] = -1;
    out_psym[0] = -1;
    slot[hash_vec(out_map, nq) & (hsize - 1)] = 0;

    /* states [head, count) are the FIFO Q_tmp; [0, head) are in Q_s */
    for (int64_t head = 0; head < count; ++head) {
        const int32_t *f = out_map + head * nq;
        for (int32_t k = 0; k < nsym; ++k) {
            uint8_t sigma = symbols[k];
            for (int32_t q = 0; q < nq; ++q)
                fnext[q] = delta[(int64_t)f[q] * 256 + sigma];
            uint64_t h = hash_vec(fnext, nq) & (hsize - 1);
            int64_t id = -1;
            while (slot[h] >= 0) {
                if (memcmp(out_map + slot[h] * nq, fnext, (size_t)nq * sizeof(int32_t)) == 0) {
                    id = slot[h];
                    break;
                }
                h = (h + 1) & (hsize - 1);
            }
            if (id < 0) {
                if (count >= cap) { free(slot); free(fnext); return -1; }
                id = count++;
                memcpy(out_map + id * nq, fnext, (size_t)nq * sizeof(int32_t));
                out_parent[id] = (int32_t)head;
                out_psym[id] = k;
                slot[h] = id;
            }
            out_delta[head * nsym + k] = (int32_t)id;
        }
    }
    free(slot);
    free(fnext);
    return count;
}

/* ------------------------------------------------------------------------
 * Alg. 5, the loop of one thread: f <- delta_s[f, sigma] from f_start over
 * the text.  sym_index maps a byte to its symbol index (-1: not in Sigma,
 * which is an error: returns -1).
 * ---------------------------------------------------------------------- */
int32_t oracle_sfa_run(const int32_t *sfa_delta, int32_t nsym, const int32_t *sym_index,
                       int32_t f_start, const uint8_t *text, uint64_t n)
{
    int32_t f = f_start;
    for (uint64_t i = 0; i < n; ++i) {
        int32_t k = sym_index[text[i]];
        if (k < 0) return -1;
        f = sfa_delta[(int64_t)f * nsym + k];
    }
    return f;
}

/* ------------------------------------------------------------------------
 * Threaded forms: each of p chunks [bounds[i], bounds[i+1]) is computed
 * independently (the "parallel" loops of Alg. 3 and Alg. 5); chunks are
 * dealt to nthreads POSIX threads round robin.
 * ---------------------------------------------------------------------- */
typedef struct {
    int kind;                 /* 3: Alg. 3, 5: Alg. 5 */
    const int32_t *table;     /* Alg. 3: DFA delta; Alg. 5: SFA delta */
    int32_t nq, nsym;
    const int32_t *sym_index;
    const uint8_t *text;
    const uint64_t *bounds;
    int32_t p, tid, nthreads;
    int32_t *out;             /* Alg. 3: [p*nq]; Alg. 5: [p] */
    int32_t status;
} chunk_job;

static void *chunk_worker(void *arg)
{
    chunk_job *j = (chunk_job *)arg;
    for (int32_t i = j->tid; i < j->p; i += j->nthreads) {
        const uint8_t *w = j->text + j->bounds[i];
        uint64_t m = j->bounds[i + 1] - j->bounds[i];
        if (j->kind == 5) {
            int32_t f = oracle_sfa_run(j->table, j->nsym, j->sym_index, 0, w, m);
            if (f < 0) j->status = -1;
            j->out[i] = f;
        } else {
            /* Alg. 3: T_i[q] <- q for all q, then T_i[q] <- delta(T_i[q], sigma) */
            int32_t *T = j->out + (int64_t)i * j->nq;
            for (int32_t q = 0; q < j->nq; ++q) T[q] = q;
            for (uint64_t s = 0; s < m; ++s)
                for (int32_t q = 0; q < j->nq; ++q)
                    T[q] = j->table[(int64_t)T[q] * 256 + w[s]];
        }
    }
    return NULL;
}

static int run_chunks(chunk_job proto, int32_t nthreads)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    chunk_job jobs[256];
    int rc = 0;
    for (int32_t t = 0; t < nthreads; ++t) {
        jobs[t] = proto;
        jobs[t].tid = t;
        jobs[t].nthreads = nthreads;
        jobs[t].status = 0;
        if (pthread_create(&th[t], NULL, chunk_worker, &jobs[t]) != 0) { rc = -2; nthreads = t; break; }
    }
    for (int32_t t = 0; t < nthreads; ++t) {
        pthread_join(th[t], NULL);
        if (jobs[t].status) rc = jobs[t].status;
    }
    return rc;
}

int oracle_alg5_chunks(const int32_t *sfa_delta, int32_t nsym, const int32_t *sym_index,
                       const uint8_t *text, const uint64_t *bounds, int32_t p,
                       int32_t *out_f, int32_t nthreads)
{
    chunk_job j;
    memset(&j, 0, sizeof j);
    j.kind = 5; j.table = sfa_delta; j.nsym = nsym; j.sym_index = sym_index;
    j.text = text; j.bounds = bounds; j.p = p; j.out = out_f;
    return run_chunks(j, nthreads);
}

int oracle_alg3_chunks(const int32_t *delta, int32_t nq, const uint8_t *text,
                       const uint64_t *bounds, int32_t p, int32_t *out_T, int32_t nthreads)
{
    chunk_job j;
    memset(&j, 0, sizeof j);
    j.kind = 3; j.table = delta; j.nq = nq;
    j.text = text; j.bounds = bounds; j.p = p; j.out = out_T;
    return run_chunks(j, nthreads);
}

/* Sequential DFA runs of p chunks from given start states (used to count
 * accepting positions chunk by chunk after a reduction). */
typedef struct {
    const int32_t *delta; const uint8_t *accept; const uint8_t *text;
    const uint64_t *bounds; const int32_t *starts; int32_t p, tid, nthreads;
    int32_t *out_final; uint64_t *out_count;
} dfa_job;

static void *dfa_worker(void *arg)
{
    dfa_job *j = (dfa_job *)arg;
    for (int32_t i = j->tid; i < j->p; i += j->nthreads)
        j->out_final[i] = oracle_dfa_run(j->delta, 0, j->starts[i], j->accept,
                                         j->text + j->bounds[i],
                                         j->bounds[i + 1] - j->bounds[i], &j->out_count[i]);
    return NULL;
}

int oracle_dfa_chunks(const int32_t *delta, const uint8_t *accept, const uint8_t *text,
                      const uint64_t *bounds, const int32_t *starts, int32_t p,
                      int32_t *out_final, uint64_t *out_count, int32_t nthreads)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    dfa_job jobs[256];
    for (int32_t t = 0; t < nthreads; ++t) {
        dfa_job j = {delta, accept, text, bounds, starts, p, t, nthreads, out_final, out_count};
        jobs[t] = j;
        if (pthread_create(&th[t], NULL, dfa_worker, &jobs[t]) != 0) { nthreads = t; break; }
    }
    for (int32_t t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    return 0;
}
