"""User-level driver of Algorithm 1 on top of the C ABI.

``RTRD`` owns one plan and the device buffers of every step (Y_n, Q_n, P,
Z_n, G_n) and calls the entry points in the order of Algorithm 1.
``decompose`` is the end-to-end call for a host tensor: copy in, run, copy
the cores out.  No arithmetic happens here.
"""
import torch

from . import rtr


class RTRD:
    def __init__(self, dims, K, R, prec="fp32", seed=0, sweeps=20, tol=1e-2, chain_order=None,
                 device="cuda", power=0, sequential=False, pair=False):
        """power: power iterations per sketch (the remark after Algorithm 1);
        sequential: the sequential projection (rtr_project_sequential) in place
        of steps 3-8; pair: a BF16 plan sketches its last two modes from the
        same tiles of X (RTR_PARAM_PAIR)."""
        self.params = rtr.make_params(prec, seed, sweeps, tol, chain_order, power,
                                      flags=rtr.PARAM_PAIR if pair else 0)
        self.sequential = bool(sequential)
        with torch.cuda.device(device):
            self.plan = rtr.rtr_plan_create(dims, K, R, self.params)
        p = self.plan
        dev = torch.device(device)
        f64 = torch.float64
        N = p.N
        self.device = dev
        self.Y = [torch.empty((d, k), dtype=f64, device=dev) if pr else None
                  for d, k, pr in zip(p.dims, p.K, p.projected)]
        self.Q = [torch.empty((d, k), dtype=f64, device=dev) for d, k in zip(p.dims, p.K)]
        self.P = torch.empty(p.K, dtype=p.x_dtype, device=dev)
        self.Z = [torch.empty((p.R[n], p.K[n], p.R[(n + 1) % N]), dtype=f64, device=dev) for n in range(N)]
        self.G = [torch.empty((p.R[n], p.dims[n], p.R[(n + 1) % N]), dtype=f64, device=dev) for n in range(N)]
        self.err = torch.zeros(max(int(sweeps), 1), dtype=f64, device=dev)
        self.rse = torch.zeros(1, dtype=f64, device=dev)
        self.ranks = list(p.R)

    # Algorithm 1, steps 3-8
    def sketch(self, X, stream=None):
        rtr.rtr_sketch(self.plan, X, self.Y, stream)

    def project(self, X, stream=None):
        rtr.rtr_project(self.plan, X, self.Y, self.Q, self.P, stream)

    # step 9
    def als(self, init=None, stream=None):
        if init is not None:
            for z, i in zip(self.Z, init):
                z.copy_(torch.as_tensor(i, dtype=torch.float64), non_blocking=True)
        rtr.rtr_als(self.plan, self.P, self.Z, init is not None, self.err, stream)

    def svd(self, tol=None, ranks=None, stream=None):
        tol = self.params.tol if tol is None else tol
        self.ranks = rtr.rtr_svd(self.plan, self.P, tol, self.Z, ranks, stream)
        return self.ranks

    # step 11
    def backproject(self, stream=None):
        rtr.rtr_backproject(self.plan, self.Z, self.Q, self.G, self.ranks, stream)

    def compute_rse(self, stream=None):
        rtr.rtr_rse(self.plan, self.P, self.Z, self.rse, self.ranks, stream)

    def project_sequential(self, X, stream=None):
        rtr.rtr_project_sequential(self.plan, X, self.Y, self.Q, self.P, stream)

    def run(self, X, method="als", init=None, ranks=None, stream=None):
        if self.sequential:
            self.project_sequential(X, stream)
        else:
            self.sketch(X, stream)
            self.project(X, stream)
        if method == "als":
            self.als(init, stream)
        elif method == "svd":
            self.svd(ranks=ranks, stream=stream)
        else:
            raise ValueError(method)
        self.backproject(stream)
        return self

    def cores(self):
        """Back-projected cores G_n (views with the chosen ranks)."""
        N = self.plan.N
        out = []
        for n in range(N):
            a, b = self.ranks[n], self.ranks[(n + 1) % N]
            out.append(self.G[n].view(-1)[: a * self.plan.dims[n] * b].view(a, self.plan.dims[n], b))
        return out

    def reconstruct(self, out_prec="fp64", stream=None):
        dims = self.plan.dims
        out = torch.empty(dims, dtype=torch.float64 if out_prec == "fp64" else torch.float32, device=self.device)
        work = torch.empty(rtr.rtr_reconstruct_work_bytes(dims, self.ranks), dtype=torch.uint8, device=self.device)
        rtr.rtr_reconstruct(dims, self.ranks, [g.contiguous() for g in self.cores()], out_prec, out, work, stream)
        return out


def decompose(X_host, K, R, method="als", prec="fp32", seed=0, sweeps=20, tol=1e-2, init=None,
              engine=None, stream=None):
    """End to end from a host tensor: H2D copy of X, Algorithm 1 on the GPU,
    D2H copy of the cores G_n and the RSE.  Reuses `engine` (an RTRD) if given."""
    eng = engine or RTRD(X_host.shape, K, R, prec, seed, sweeps, tol)
    Xd = X_host.to(eng.device, non_blocking=True)
    eng.run(Xd, method, init, stream=stream)
    eng.compute_rse(stream)
    G = [g.to("cpu", non_blocking=True) for g in eng.cores()]
    rse = eng.rse.to("cpu", non_blocking=True)
    torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
    return G, float(rse[0]), eng


def decompose_stream(X_hosts, K, R, method="als", prec="fp32", seed=0, sweeps=20, tol=1e-2, init=None,
                     engines=None, inflight=2):
    """End to end for a sequence of host tensors of one shape: per tensor the
    H2D copy of X, Algorithm 1 on the GPU, and the D2H copies of the cores G_n
    and the RSE.  Consecutive tensors alternate over `inflight` engines (each
    its own plan, device copy of X and stream), so that one tensor's copies
    and TR-ALS overlap the next one's sketch.  Page-locked host tensors let
    the copies run asynchronously.  `engines`: RTRD objects to reuse (one per
    tensor in flight).  Returns [(G, rse)] in input order."""
    if not X_hosts:
        return []
    dims = tuple(X_hosts[0].shape)
    engs = list(engines) if engines is not None else \
        [RTRD(dims, K, R, prec, seed, sweeps, tol) for _ in range(max(1, inflight))]
    n = len(engs)
    streams = [torch.cuda.Stream(e.device) for e in engs]
    bufs = [torch.empty(dims, dtype=e.plan.x_dtype, device=e.device) for e in engs]
    main = torch.cuda.current_stream(engs[0].device)
    for st in streams:
        st.wait_stream(main)
    out = []
    for i, Xh in enumerate(X_hosts):
        k = i % n
        eng, st, Xd = engs[k], streams[k], bufs[k]
        with torch.cuda.stream(st):
            Xd.copy_(Xh, non_blocking=True)
            eng.run(Xd, method, init, stream=st)
            eng.compute_rse(st)
            G = [torch.empty(g.shape, dtype=g.dtype, pin_memory=True) for g in eng.cores()]
            for g, gd in zip(G, eng.cores()):
                g.copy_(gd, non_blocking=True)
            rse = torch.empty(1, dtype=torch.float64, pin_memory=True)
            rse.copy_(eng.rse, non_blocking=True)
        out.append((G, rse))
    for st in streams:
        st.synchronize()
    return [(G, float(r[0])) for G, r in out]
