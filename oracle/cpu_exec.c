/*
 * Threaded CPU execution of the synchronization workloads.
 * ORACLE -- TEST INFRASTRUCTURE ONLY: called by the tests and by the CPU-baseline leg of the
 * benchmark, never by the CUDA library, and sharing no code with it.
 *
 * Each workload runs with real locks on host threads using C11 sequentially consistent
 * atomics, following the algorithms of Section 5 ("Design") of Stuart & Owens, "Efficient
 * Synchronization Primitives for GPUs":
 *   mutex kinds   0 spin lock on compare-and-swap          (Algorithm 1, spin-lock mutex)
 *                 1 spin lock with exponential backoff     (spin-lock mutex, UseBackoff)
 *                 2 fetch-and-add ticket lock              (FA mutex)
 *                 3 queue lock, one flag slot per waiter   (sleep-waiting queue lock)
 *   semaphores    0 sleeping (FA) semaphore, 1 spin-lock semaphore, 2 spin-lock + backoff
 *   barriers      0 two-stage atomic counter, 1 decentralized flag barrier (XF)
 * A "block" of the GPU workload is one unit of work here; the mutex and semaphore runs map
 * blocks round-robin onto `nthreads` host threads (thread t runs blocks t, t+T, ...; each
 * block's acquisitions stay in program order), while a barrier run needs one thread per
 * block.  Busy waits call sched_yield() after a while so oversubscribed runs still progress.
 * The final states these runs produce must equal the plain definitions in calc.py.
 */
#include <pthread.h>
#include <sched.h>
#include <stdatomic.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

#define LINE 128
#define GOLDEN32 0x9E3779B1u

typedef struct { _Alignas(LINE) atomic_uint v; char pad[LINE - sizeof(atomic_uint)]; } line_t;

static double now_s(void) {
  struct timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

static void spin_iters(uint32_t n) {
  volatile uint32_t sink = 0;
  for (uint32_t i = 0; i < n; ++i) sink += i;
}

/* One unit of waiting: after 256 polls yield the core to another thread. */
static void wait_tick(uint32_t* polls) {
  if (++*polls >= 256) { *polls = 0; sched_yield(); }
}

static uint32_t lowbias32(uint32_t x) {
  x ^= x >> 16; x *= 0x7feb352du; x ^= x >> 15; x *= 0x846ca68bu; x ^= x >> 16;
  return x;
}

static uint32_t rotl32(uint32_t x, int k) { return (x << k) | (x >> (32 - k)); }

/* ------------------------------------------------------------------------------------ */
/* Mutex workload                                                                       */
/* ------------------------------------------------------------------------------------ */

typedef struct {
  line_t lock;    /* CAS kinds: 0 free, 1 held */
  line_t ticket;  /* ticket kinds: next ticket to hand out */
  line_t turn;    /* ticket lock: ticket now allowed in */
  line_t* flags;  /* queue lock: q slots */
  uint32_t q;
} cpu_mutex;

typedef struct {
  cpu_mutex* m;
  int kind, nblocks, acq, cs_words, nthreads, tid;
  uint32_t backoff_max;
  const uint32_t *addend, *delay;
  uint32_t *data, *total, *log, *ticket, *count;
  atomic_int* go;
} mutex_job;

static uint32_t mutex_lock(cpu_mutex* m, int kind, uint32_t backoff_max) {
  uint32_t polls = 0;
  if (kind == 0 || kind == 1) {
    uint32_t d = 16;
    for (;;) {
      unsigned expect = 0;
      if (atomic_compare_exchange_strong(&m->lock.v, &expect, 1u)) return 0xFFFFFFFFu;
      if (kind == 1) { spin_iters(d); d = d * 2 > backoff_max ? backoff_max : d * 2; }
      wait_tick(&polls);
    }
  }
  if (kind == 2) {
    uint32_t t = atomic_fetch_add(&m->ticket.v, 1u);
    while (atomic_load(&m->turn.v) != t) wait_tick(&polls);
    return t;
  }
  uint32_t t = atomic_fetch_add(&m->ticket.v, 1u);
  while (atomic_load(&m->flags[t & (m->q - 1)].v) != t) wait_tick(&polls);
  return t;
}

static void mutex_unlock(cpu_mutex* m, int kind, uint32_t t) {
  if (kind == 0 || kind == 1) atomic_store(&m->lock.v, 0u);
  else if (kind == 2) atomic_store(&m->turn.v, t + 1u);
  else atomic_store(&m->flags[(t + 1u) & (m->q - 1)].v, t + 1u);
}

static void* mutex_worker(void* p) {
  mutex_job* j = (mutex_job*)p;
  const uint32_t n = (uint32_t)j->nblocks * (uint32_t)j->acq;
  while (!atomic_load(j->go)) {}
  for (int a = 0; a < j->acq; ++a) {
    for (int b = j->tid; b < j->nblocks; b += j->nthreads) {
      const uint32_t id = (uint32_t)b * (uint32_t)j->acq + (uint32_t)a;
      if (j->delay) spin_iters(j->delay[id]);
      uint32_t t = mutex_lock(j->m, j->kind, j->backoff_max);
      uint32_t seq = *j->total;
      *j->total = seq + 1u;
      if (seq < n) j->log[seq] = id;
      j->ticket[id] = t;
      const uint32_t v = j->addend[id];
      for (int i = 0; i < j->cs_words; ++i) j->data[i] += v ^ ((uint32_t)i * GOLDEN32);
      mutex_unlock(j->m, j->kind, t);
      j->count[b] += 1u;
    }
  }
  return NULL;
}

/* Runs the mutex workload; returns 0 on success.  Outputs must be zeroed by the caller. */
int oracle_mutex_run(int kind, int nblocks, int acq, int cs_words, int nthreads,
                     const uint32_t* addend, const uint32_t* delay, uint32_t* data,
                     uint32_t* total, uint32_t* log, uint32_t* ticket, uint32_t* count,
                     double* seconds) {
  if (kind < 0 || kind > 3 || nblocks <= 0 || acq < 0 || cs_words < 0 || nthreads <= 0) return 1;
  if (nthreads > nblocks) nthreads = nblocks;
  cpu_mutex m;
  memset(&m, 0, sizeof m);
  uint32_t q = 1;
  while (q < (uint32_t)nthreads) q <<= 1;
  m.q = q;
  m.flags = (line_t*)aligned_alloc(LINE, sizeof(line_t) * q);
  if (!m.flags) return 2;
  for (uint32_t i = 0; i < q; ++i) atomic_init(&m.flags[i].v, i == 0 ? 0u : i - q);
  atomic_init(&m.lock.v, 0u); atomic_init(&m.ticket.v, 0u); atomic_init(&m.turn.v, 0u);
  atomic_int go; atomic_init(&go, 0);
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nthreads);
  mutex_job* jobs = (mutex_job*)malloc(sizeof(mutex_job) * (size_t)nthreads);
  if (!th || !jobs) { free(m.flags); free(th); free(jobs); return 2; }
  for (int t = 0; t < nthreads; ++t) {
    mutex_job jb = {&m, kind, nblocks, acq, cs_words, nthreads, t, 1u << 12,
                    addend, delay, data, total, log, ticket, count, &go};
    jobs[t] = jb;
    pthread_create(&th[t], NULL, mutex_worker, &jobs[t]);
  }
  double t0 = now_s();
  atomic_store(&go, 1);
  for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
  *seconds = now_s() - t0;
  free(m.flags); free(th); free(jobs);
  return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Counting-semaphore workload                                                          */
/* ------------------------------------------------------------------------------------ */

typedef struct {
  line_t count, ticket, turn;  /* sleeping semaphore */
  line_t s;                    /* spin-lock semaphore: X + 1, 0 = internally locked */
  line_t occ, max_occ;
  int n;
} cpu_sem;

typedef struct {
  cpu_sem* s;
  int kind, nblocks, pairs, nthreads, tid;
  const uint32_t *hold, *addend;
  uint32_t *count, *total;
  atomic_uint* tally;
  atomic_int* go;
} sem_job;

static void sem_wait(cpu_sem* s, int kind) {
  uint32_t polls = 0;
  if (kind == 0) {
    int old = (int)atomic_fetch_add(&s->count.v, 1u);
    if (old < s->n) return;
    uint32_t w = atomic_fetch_add(&s->ticket.v, 1u);
    while ((int32_t)(atomic_load(&s->turn.v) - w) <= 0) wait_tick(&polls);
    return;
  }
  uint32_t d = 16;
  for (;;) {
    uint32_t v = atomic_exchange(&s->s.v, 0u);
    if (v > 1) { atomic_exchange(&s->s.v, v - 1u); return; }
    if (v == 1) atomic_exchange(&s->s.v, 1u);
    if (kind == 2) { spin_iters(d); d = d * 2 > 4096 ? 4096 : d * 2; }
    wait_tick(&polls);
  }
}

static void sem_post(cpu_sem* s, int kind) {
  uint32_t polls = 0;
  if (kind == 0) {
    int old = (int)atomic_fetch_sub(&s->count.v, 1u);
    if (old > s->n) atomic_fetch_add(&s->turn.v, 1u);
    return;
  }
  for (;;) {
    uint32_t v = atomic_exchange(&s->s.v, 0u);
    if (v > 0) { atomic_exchange(&s->s.v, v + 1u); return; }
    wait_tick(&polls);
  }
}

static void* sem_worker(void* p) {
  sem_job* j = (sem_job*)p;
  while (!atomic_load(j->go)) {}
  for (int k = 0; k < j->pairs; ++k) {
    for (int b = j->tid; b < j->nblocks; b += j->nthreads) {
      const uint32_t id = (uint32_t)b * (uint32_t)j->pairs + (uint32_t)k;
      sem_wait(j->s, j->kind);
      uint32_t o = atomic_fetch_add(&j->s->occ.v, 1u) + 1u;
      uint32_t m = atomic_load(&j->s->max_occ.v);
      while (o > m && !atomic_compare_exchange_weak(&j->s->max_occ.v, &m, o)) {}
      if (j->s->n == 1) *j->total += 1u;
      if (j->hold) spin_iters(j->hold[id]);
      atomic_fetch_add(j->tally, j->addend[id]);
      atomic_fetch_sub(&j->s->occ.v, 1u);
      sem_post(j->s, j->kind);
      j->count[b] += 1u;
    }
  }
  return NULL;
}

int oracle_sem_run(int kind, int nblocks, int pairs, int n_init, int nthreads,
                   const uint32_t* hold, const uint32_t* addend, uint32_t* count,
                   uint32_t* total, uint32_t* tally, uint32_t* max_occ, double* seconds) {
  if (kind < 0 || kind > 2 || nblocks <= 0 || pairs < 0 || n_init <= 0 || nthreads <= 0) return 1;
  if (nthreads > nblocks) nthreads = nblocks;
  cpu_sem* s = (cpu_sem*)aligned_alloc(LINE, sizeof(cpu_sem) + LINE);
  if (!s) return 2;
  memset(s, 0, sizeof *s);
  atomic_init(&s->count.v, 0u); atomic_init(&s->ticket.v, 0u); atomic_init(&s->turn.v, 0u);
  atomic_init(&s->s.v, (uint32_t)n_init + 1u);
  atomic_init(&s->occ.v, 0u); atomic_init(&s->max_occ.v, 0u);
  s->n = n_init;
  atomic_uint tal; atomic_init(&tal, 0u);
  atomic_int go; atomic_init(&go, 0);
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nthreads);
  sem_job* jobs = (sem_job*)malloc(sizeof(sem_job) * (size_t)nthreads);
  if (!th || !jobs) { free(s); free(th); free(jobs); return 2; }
  for (int t = 0; t < nthreads; ++t) {
    sem_job jb = {s, kind, nblocks, pairs, nthreads, t, hold, addend, count, total, &tal, &go};
    jobs[t] = jb;
    pthread_create(&th[t], NULL, sem_worker, &jobs[t]);
  }
  double t0 = now_s();
  atomic_store(&go, 1);
  for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
  *seconds = now_s() - t0;
  *tally = atomic_load(&tal);
  *max_occ = atomic_load(&s->max_occ.v);
  free(s); free(th); free(jobs);
  return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Barrier workload                                                                     */
/* ------------------------------------------------------------------------------------ */

typedef struct {
  line_t count, release;  /* atomic barrier */
  line_t* arrive;         /* flag barrier: one flag per block */
  line_t* rel;            /* flag barrier: one release flag per block */
  uint32_t* slot;         /* [2][nblocks] */
  int kind, nblocks, rounds, full;
  uint32_t *chk, *mix, *bad;
  atomic_int go;
} cpu_bar;

typedef struct { cpu_bar* b; int id; } bar_job;

static void barrier_cross(cpu_bar* B, int id, uint32_t* epoch) {
  uint32_t polls = 0;
  const uint32_t e = *epoch + 1u;
  if (B->kind == 0) {
    uint32_t old = atomic_fetch_add(&B->count.v, 1u);
    if (old == (uint32_t)B->nblocks - 1u) {
      atomic_store(&B->count.v, 0u);
      atomic_store(&B->release.v, e);
    } else {
      while (atomic_load(&B->release.v) != e) wait_tick(&polls);
    }
  } else {
    atomic_store(&B->arrive[id].v, e);
    if (id == 0) {
      for (int j = 1; j < B->nblocks; ++j)
        while (atomic_load(&B->arrive[j].v) != e) wait_tick(&polls);
      for (int j = 1; j < B->nblocks; ++j) atomic_store(&B->rel[j].v, e);
    } else {
      while (atomic_load(&B->rel[id].v) != e) wait_tick(&polls);
    }
  }
  *epoch = e;
}

static void* bar_worker(void* p) {
  bar_job* jb = (bar_job*)p;
  cpu_bar* B = jb->b;
  const int b = jb->id;
  const uint32_t nb = (uint32_t)B->nblocks;
  uint32_t epoch = 0, mix = 0, bad = 0;
  while (!atomic_load(&B->go)) {}
  for (int r = 0; r < B->rounds; ++r) {
    uint32_t* buf = B->slot + (size_t)(r & 1) * nb;
    buf[b] = (uint32_t)r * nb + (uint32_t)b;
    barrier_cross(B, b, &epoch);
    if (B->full) {
      uint32_t x = 0, s = 0;
      for (uint32_t j = 0; j < nb; ++j) {
        const uint32_t v = buf[j];
        x ^= v;
        s += lowbias32(v);
        bad += v != (uint32_t)r * nb + j;
      }
      B->chk[(size_t)r * nb + (size_t)b] = x;
      mix = rotl32(mix, 5) ^ s;
    } else {
      const uint32_t p2 = ((uint32_t)b + (uint32_t)r + 1u) % nb;
      const uint32_t v = buf[p2];
      mix = rotl32(mix, 5) ^ lowbias32(v);
      bad += v != (uint32_t)r * nb + p2;
    }
  }
  B->mix[b] = mix;
  B->bad[b] = bad;
  return NULL;
}

/* Runs the barrier workload with one thread per block (full=1: every block reads every slot;
 * full=0: one partner slot per round).  chk may be NULL when full=0. */
int oracle_barrier_run(int kind, int nblocks, int rounds, int full, uint32_t* chk,
                       uint32_t* mix, uint32_t* bad, double* seconds) {
  if (kind < 0 || kind > 1 || nblocks <= 0 || rounds < 0) return 1;
  if (full && !chk) return 1;
  cpu_bar* B = (cpu_bar*)aligned_alloc(LINE, sizeof(cpu_bar) + LINE);
  if (!B) return 2;
  memset(B, 0, sizeof *B);
  B->arrive = (line_t*)aligned_alloc(LINE, sizeof(line_t) * (size_t)nblocks);
  B->rel = (line_t*)aligned_alloc(LINE, sizeof(line_t) * (size_t)nblocks);
  B->slot = (uint32_t*)calloc(2 * (size_t)nblocks, sizeof(uint32_t));
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nblocks);
  bar_job* jobs = (bar_job*)malloc(sizeof(bar_job) * (size_t)nblocks);
  if (!B->arrive || !B->rel || !B->slot || !th || !jobs) return 2;
  for (int j = 0; j < nblocks; ++j) { atomic_init(&B->arrive[j].v, 0u); atomic_init(&B->rel[j].v, 0u); }
  atomic_init(&B->count.v, 0u); atomic_init(&B->release.v, 0u); atomic_init(&B->go, 0);
  B->kind = kind; B->nblocks = nblocks; B->rounds = rounds; B->full = full;
  B->chk = chk; B->mix = mix; B->bad = bad;
  for (int j = 0; j < nblocks; ++j) {
    jobs[j].b = B; jobs[j].id = j;
    pthread_create(&th[j], NULL, bar_worker, &jobs[j]);
  }
  double t0 = now_s();
  atomic_store(&B->go, 1);
  for (int j = 0; j < nblocks; ++j) pthread_join(th[j], NULL);
  *seconds = now_s() - t0;
  free(B->arrive); free(B->rel); free(B->slot); free(th); free(jobs); free(B);
  return 0;
}
