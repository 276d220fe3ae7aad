"""Training driver of the learned initial guess (argument marshalling around the C ABI).

Pairs are recorded from the library's own solver: before a step the previous coarse
increment q = Phi_c^n is copied out, after it the coarse right-hand side r of Eq. 23 and
the converged Phi_c^{n+1} (the target).  Training runs the library's CUDA forward,
backward and Adam kernels (cgp_mlp_train_step); PyTorch only holds the device buffers.
"""

import numpy as np

from . import binding as cg


class PairStore:
    """Device buffers of recorded (r, q, target) triples on one mesh level."""

    def __init__(self, n, capacity):
        import torch
        self.n, self.cap, self.count = n, capacity, 0
        self.r = torch.empty((capacity, n), dtype=torch.float64, device="cuda")
        self.q = torch.empty_like(self.r)
        self.t = torch.empty_like(self.r)

    def record(self, solver, steps):
        """Advance `steps` steps of `solver` (a binding.Solver), storing one triple per step."""
        k = self.count
        m = min(steps, self.cap - k)
        if m > 0:
            cg.cgp_record_pairs(solver.handle, m, self.r[k:k + m], self.q[k:k + m], self.t[k:k + m])
            self.count += m
        return self.count


def train(net, store, iters, batch=8, lr=1e-3, seed=0, log_every=0):
    """Adam on random batches of the store; returns the loss history (every log_every, and last)."""
    import torch
    rng = np.random.default_rng(seed)
    n = store.n
    rb = torch.empty((batch, n), dtype=torch.float64, device="cuda")
    qb, tb = torch.empty_like(rb), torch.empty_like(rb)
    hist = []
    for it in range(iters):
        idx = torch.as_tensor(rng.integers(0, store.count, size=batch), device="cuda")
        torch.index_select(store.r[:store.count], 0, idx, out=rb)
        torch.index_select(store.q[:store.count], 0, idx, out=qb)
        torch.index_select(store.t[:store.count], 0, idx, out=tb)
        want = (log_every and it % log_every == 0) or it == iters - 1
        loss = cg.cgp_mlp_train_step(net, rb, qb, tb, batch, lr, want_loss=want)
        if want:
            hist.append((it, loss))
    return hist


def mean_loss(net, store, batch=8):
    """Mean training loss over every stored triple (the library's forward pass and loss)."""
    tot, cnt = 0.0, 0
    for k0 in range(0, store.count, batch):
        b = min(batch, store.count - k0)
        loss, _ = cg.cgp_mlp_grad(net, store.r[k0:k0 + b], store.q[k0:k0 + b], store.t[k0:k0 + b], b)
        tot += loss * b
        cnt += b
    return tot / max(cnt, 1)


def init_params(seed=0):
    """He-style initialisation of the parameter vector (last layer small so that the
    initial prediction stays close to the previous increment)."""
    rng = np.random.default_rng(seed)
    p = np.zeros(cg.cgp_mlp_param_count(), np.float32)
    o = 0
    for fin, fout, scale in ((4, 64, 1.0), (64, 64, 1.0), (64, 1, 0.01)):
        w = rng.standard_normal((fout, 2 * fin)) * np.sqrt(2.0 / (2 * fin)) * scale
        p[o:o + w.size] = w.ravel()
        o += w.size + fout          # biases stay zero
    return p


class MultiMeshTrainer:
    """One network trained on pairs recorded on several meshes: one cgp_mlp per mesh level
    (each owns that level's adjacency and activation buffers); before every Adam step the
    weights and the Adam state move to the network of the mesh the batch comes from
    (cgp_mlp_copy_state), so the sequence of steps is that of a single network."""

    def __init__(self, params, batch=8):
        self.batch = batch
        self.params = params
        self.nets, self.stores = [], []
        self.current = None

    def add(self, mesh_handle, level, store):
        net = cg.cgp_mlp_create(mesh_handle, level, self.batch)
        cg.cgp_mlp_set_params(net, self.params)
        self.nets.append(net)
        self.stores.append(store)
        if self.current is None:
            self.current = 0

    def train(self, iters, lr=1e-3, seed=0, log_every=0):
        """Adam steps on random batches; a batch's mesh is drawn in proportion to its pairs."""
        import torch
        rng = np.random.default_rng(seed)
        counts = np.array([s.count for s in self.stores], dtype=np.float64)
        prob = counts / counts.sum()
        bufs = {}
        hist = []
        for it in range(iters):
            k = int(rng.choice(len(self.stores), p=prob))
            st = self.stores[k]
            if k != self.current:
                cg.cgp_mlp_copy_state(self.nets[k], self.nets[self.current])
                self.current = k
            if st.n not in bufs:
                rb = torch.empty((self.batch, st.n), dtype=torch.float64, device="cuda")
                bufs[st.n] = (rb, torch.empty_like(rb), torch.empty_like(rb))
            rb, qb, tb = bufs[st.n]
            idx = torch.as_tensor(rng.integers(0, st.count, size=self.batch), device="cuda")
            torch.index_select(st.r[:st.count], 0, idx, out=rb)
            torch.index_select(st.q[:st.count], 0, idx, out=qb)
            torch.index_select(st.t[:st.count], 0, idx, out=tb)
            want = (log_every and it % log_every == 0) or it == iters - 1
            loss = cg.cgp_mlp_train_step(self.nets[k], rb, qb, tb, self.batch, lr, want_loss=want)
            if want:
                hist.append((it, k, loss))
        return hist

    def get_params(self):
        return cg.cgp_mlp_get_params(self.nets[self.current])

    def close(self):
        for net in self.nets:
            cg.cgp_mlp_destroy(net)
        self.nets = []
