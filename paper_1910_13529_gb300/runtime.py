"""PyTorch plumbing around the C ABI: device tensors for fields and particles, the caller's
CUDA stream, and host copies for inspection.  No PIC arithmetic happens here."""
import ctypes

import numpy as np
import torch

from . import (PIC_FILTER_5PASS, PIC_FILTER_NONE, PIC_SOLVER_CUSTOM, PIC_SOLVER_KT, PIC_SOLVER_PSATD,
               PIC_SOLVER_SPECTRAL, PIC_SOLVER_YEE, encode_cells, pic_batch_create, pic_batch_destroy,
               pic_batch_instance, pic_batch_step, pic_bind_fields, pic_bind_species,
               pic_config, pic_create, pic_deposit, pic_destroy, pic_diag, pic_field_advance,
               pic_autotune, pic_gather_push, pic_gauss, pic_get_coefficients, pic_get_count, pic_get_state,
               pic_filter_current, pic_get_tuning, pic_rho, pic_sort, pic_step, pic_sync)


def make_config(ndim, nz, nx, ny=1, dz=1.0, dx=1.0, dy=1.0, dt=0.5, solver="yee", M=16, coef=None,
                fit_wk=0.0, fit_n=0.0, shape=1, moving_window=False, inject_species=-1,
                inject_ppc=(1, 1, 1), rho_bg=0.0, sort_every=0, current_filter=False, coef_b=None):
    c = pic_config()
    c.ndim, c.nz, c.nx, c.ny = int(ndim), int(nz), int(nx), int(ny if ndim == 3 else 1)
    c.dz, c.dx, c.dy, c.dt = float(dz), float(dx), float(dy), float(dt)
    solvers = {"yee": PIC_SOLVER_YEE, "custom": PIC_SOLVER_CUSTOM, "spectral": PIC_SOLVER_SPECTRAL,
               "kt": PIC_SOLVER_KT, "psatd": PIC_SOLVER_PSATD}
    if solver not in solvers:
        raise ValueError(f"solver {solver!r}: one of {sorted(solvers)}")
    c.solver = solvers[solver]
    c.M = int(M if solver == "custom" else 1)
    keep = None
    if coef is not None:
        keep = np.ascontiguousarray(coef, dtype=np.float64)
        c.coef = keep.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        c.M = len(keep)
    c.fit_wk, c.fit_n = float(fit_wk), float(fit_n)
    c.shape = int(shape)
    c.moving_window = int(bool(moving_window))
    c.inject_species = int(inject_species)
    for i in range(3):
        c.inject_ppc[i] = int(inject_ppc[i]) if i < len(inject_ppc) else 1
    c.rho_bg = float(rho_bg)
    c.sort_every = int(sort_every)
    c.current_filter = PIC_FILTER_5PASS if current_filter else PIC_FILTER_NONE
    if coef_b is not None:
        # the E-side and B-side sets share M: pad the shorter one with zeros (without coef the
        # library refuses coef_b)
        cb_in = np.asarray(coef_b, dtype=np.float64)
        M = max(len(keep) if keep is not None else 0, len(cb_in))
        cb = np.zeros(M)
        cb[: len(cb_in)] = cb_in
        ce = None
        if keep is not None:
            ce = np.zeros(M)
            ce[: len(keep)] = keep
            c.coef = ce.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        c.coef_b = cb.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        c.M = M
        keep = (ce, cb)
    return c, keep


class Simulation:
    """One libpic handle with its fields and species held in torch CUDA tensors."""

    def __init__(self, device="cuda:0", handle=None, **cfg):
        if not torch.cuda.is_available():
            raise RuntimeError("libpic needs a CUDA device")
        self.device = torch.device(device)
        torch.cuda.set_device(self.device)
        self.cfg = dict(cfg)
        c, keep = make_config(**cfg)
        self._c, self._keep = c, keep
        self.owned = handle is None
        self.h = pic_create(c) if handle is None else handle
        self.ndim, self.nz, self.nx, self.ny = c.ndim, c.nz, c.nx, c.ny
        shp = (3, self.ny, self.nx, self.nz)
        self.E = torch.zeros(shp, dtype=torch.float32, device=self.device)
        self.B = torch.zeros(shp, dtype=torch.float32, device=self.device)
        self.J = torch.zeros(shp, dtype=torch.float32, device=self.device)
        pic_bind_fields(self.h, self.E.data_ptr(), self.B.data_ptr(), self.J.data_ptr())
        self.species = {}

    @property
    def stream(self):
        return ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)

    def add_species(self, s, iz, ix, iy, off, u, q, m, w, cap=None, ids=None):
        n = len(iz)
        cap = max(int(cap if cap is not None else n), 1)
        cell = torch.full((cap,), -1, dtype=torch.int32, device=self.device)
        offt = torch.zeros((self.ndim, cap), dtype=torch.float32, device=self.device)
        ut = torch.zeros((3, cap), dtype=torch.float32, device=self.device)
        idt = None
        if n:
            cell[:n] = torch.from_numpy(encode_cells(iz, ix, iy, self.nz, self.nx)).to(self.device)
            offt[:, :n] = torch.from_numpy(np.ascontiguousarray(off[: self.ndim], dtype=np.float32)).to(self.device)
            ut[:, :n] = torch.from_numpy(np.ascontiguousarray(u, dtype=np.float32)).to(self.device)
        if ids is not None:
            idt = torch.full((cap,), -1, dtype=torch.int32, device=self.device)
            if n:
                idt[:n] = torch.from_numpy(np.asarray(ids, dtype=np.int32)).to(self.device)
        torch.cuda.synchronize(self.device)
        pic_bind_species(self.h, s, cell.data_ptr(), offt.data_ptr(), ut.data_ptr(),
                         idt.data_ptr() if idt is not None else None, n, cap, q, m, w)
        self.species[s] = dict(cell=cell, off=offt, u=ut, id=idt, q=q, m=m, w=w, cap=cap)

    # ---- the step ----
    def gather_push(self):
        pic_gather_push(self.h, self.stream)

    def deposit(self):
        pic_deposit(self.h, self.stream)

    def field_advance(self):
        pic_field_advance(self.h, self.stream)

    def step(self, n=1):
        pic_step(self.h, n, self.stream)

    def sort(self):
        pic_sort(self.h, self.stream)

    def filter_current(self):
        """The 5-pass current filter along z, once, in place on J (pic_filter_current)."""
        pic_filter_current(self.h, self.stream)

    def autotune(self):
        """Pick the fastest field-advance tile shape for this grid (pic_autotune)."""
        pic_autotune(self.h, self.stream)
        return pic_get_tuning(self.h)

    # ---- diagnostics ----
    def diag(self):
        return pic_diag(self.h, self.stream)

    def rho(self):
        r = torch.empty((self.ny, self.nx, self.nz), dtype=torch.float64, device=self.device)
        pic_rho(self.h, r.data_ptr(), self.stream)
        return r

    def gauss(self):
        G = torch.empty((self.ny, self.nx, self.nz), dtype=torch.float64, device=self.device)
        pic_gauss(self.h, G.data_ptr(), self.stream)
        return G

    def count(self, s):
        return pic_get_count(self.h, s, self.stream)

    def state(self):
        return pic_get_state(self.h)

    def coefficients(self):
        return pic_get_coefficients(self.h)

    def sync(self):
        pic_sync(self.h, self.stream)

    def save(self, path):
        """Checkpoint: fields, particle arrays and the run counters, to a host file."""
        from . import pic_get_next_id
        step, shifts, pending = self.state()
        sp = {s: {k: (v.cpu() if torch.is_tensor(v) else v) for k, v in d.items()} | {"n": self.count(s)}
              for s, d in self.species.items()}
        torch.save({"E": self.E.cpu(), "B": self.B.cpu(), "J": self.J.cpu(), "species": sp, "step": step,
                    "shifts": shifts, "pending": pending, "next_id": pic_get_next_id(self.h)}, path)

    def load(self, path):
        """Resume from save(): same configuration, arrays and counters restored."""
        from . import pic_set_state
        d = torch.load(path, weights_only=False)
        self.E.copy_(d["E"])
        self.B.copy_(d["B"])
        self.J.copy_(d["J"])
        for s, q in d["species"].items():
            dev = {k: (v.to(self.device) if torch.is_tensor(v) else v) for k, v in q.items()}
            self.species[s] = {k: dev[k] for k in ("cell", "off", "u", "id", "q", "m", "w", "cap")}
            pic_bind_species(self.h, s, dev["cell"].data_ptr(), dev["off"].data_ptr(), dev["u"].data_ptr(),
                             dev["id"].data_ptr() if dev["id"] is not None else None, q["n"], q["cap"], q["q"],
                             q["m"], q["w"])
        pic_set_state(self.h, d["step"], d["shifts"], d["pending"], d["next_id"])

    def particles(self, s):
        """Host copy of slots [0, count) of species s: cell, off (ndim, n), u (3, n), id."""
        n = self.count(s)
        d = self.species[s]
        out = dict(cell=d["cell"][:n].cpu().numpy(), off=d["off"][:, :n].cpu().numpy(),
                   u=d["u"][:, :n].cpu().numpy())
        out["id"] = d["id"][:n].cpu().numpy() if d["id"] is not None else None
        return out

    def close(self):
        if self.h is not None:
            torch.cuda.synchronize(self.device)
            if self.owned:
                pic_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """A libpic batch: many independent runs advanced together (pic_batch_step).  Each instance
    is a Simulation view over the batch's instance handle."""

    def __init__(self, cfgs, device="cuda:0"):
        self.device = torch.device(device)
        torch.cuda.set_device(self.device)
        made = [make_config(**c) for c in cfgs]
        self._keep = made
        self.b = pic_batch_create([m[0] for m in made])
        self.instances = [Simulation(device=device, handle=pic_batch_instance(self.b, i), **cfgs[i])
                          for i in range(len(cfgs))]

    def step(self, n=1):
        pic_batch_step(self.b, n, ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream))

    def close(self):
        if self.b is not None:
            torch.cuda.synchronize(self.device)
            for s in self.instances:
                s.h = None
            pic_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class StencilLoss:
    """Field energy left behind a rigidly moving beam after `nsteps`, as a function of the axial
    stencil coefficients C, with its gradient from the hand-written adjoint (pic_adjoint_step).

    With grid["current_filter"] the 5-pass current filter runs in every step; it precedes the
    correction and does not depend on C, so the adjoint step is unchanged.
    The particles are held rigid (their momenta never change) by giving them an effectively
    infinite mass; the loss is (1/2) sum (E^2 + B^2) dV over the cells with z index below
    (beam z index - behind).  The forward pass keeps a checkpoint (fields and particles) every
    `every` steps; the backward pass replays each segment from its checkpoint, keeping the fields
    and currents of every step of the segment, and runs the adjoint steps in reverse."""

    RIGID_MASS = 1e30

    def __init__(self, grid, species, nsteps, every=50, behind=2, device="cuda:0"):
        self.grid = dict(grid)
        self.species = species
        self.nsteps, self.every, self.behind = int(nsteps), int(every), int(behind)
        self.device = torch.device(device)

    def _sim(self, C):
        kw = {k: self.grid[k] for k in ("ndim", "nz", "nx", "ny", "dz", "dx", "dy", "dt", "shape", "current_filter")
              if k in self.grid}
        sim = Simulation(device=str(self.device), solver="custom", coef=np.asarray(C, dtype=np.float64), **kw)
        for s, sp in enumerate(self.species):
            sim.add_species(s, sp["iz"], sp["ix"], sp["iy"], sp["off"], sp["u"], sp["q"], self.RIGID_MASS, sp["w"])
        return sim

    def _mask_z(self, sim):
        """z index below which the loss is taken: the beam's lowest cell minus `behind`."""
        zmin = None
        for s in sim.species:
            cell = sim.species[s]["cell"][: sim.count(s)].cpu().numpy()
            iz = cell[cell >= 0] % (sim.nz + 2) - 1
            zmin = int(iz.min()) if zmin is None else min(zmin, int(iz.min()))
        return max(zmin - self.behind, 0)

    def _loss(self, sim, zc):
        dV = sim.cfg["dz"] * sim.cfg["dx"] * (sim.cfg.get("dy", 1.0) if sim.ndim == 3 else 1.0)
        E = sim.E[..., :zc].double()
        B = sim.B[..., :zc].double()
        return 0.5 * float((E ** 2).sum() + (B ** 2).sum()) * dV, dV

    def loss(self, C):
        sim = self._sim(C)
        sim.step(self.nsteps)
        L, _ = self._loss(sim, self._mask_z(sim))
        sim.close()
        return L

    def loss_and_grad(self, C):
        from . import pic_adjoint_step
        sim = self._sim(C)
        ckpt = []
        # forward in runs of `every` steps (an even run ends in the bound field arrays: no copy back)
        for n0 in range(0, self.nsteps, self.every):
            ckpt.append((n0, sim.E.clone(), sim.B.clone(),
                         {s: {k: sim.species[s][k].clone() for k in ("cell", "off", "u")} for s in sim.species}))
            sim.step(min(self.every, self.nsteps - n0))
        zc = self._mask_z(sim)
        L, dV = self._loss(sim, zc)
        aE = torch.zeros_like(sim.E)
        aB = torch.zeros_like(sim.B)
        aE[..., :zc] = sim.E[..., :zc] * dV
        aB[..., :zc] = sim.B[..., :zc] * dV
        grad = torch.zeros(len(C), dtype=torch.float64, device=self.device)
        stream = sim.stream
        for n0, E0, B0, parts in reversed(ckpt):
            n1 = min(n0 + self.every, self.nsteps)
            sim.E.copy_(E0)
            sim.B.copy_(B0)
            for s, arrs in parts.items():
                for k, v in arrs.items():
                    sim.species[s][k].copy_(v)
            saved = []
            for _ in range(n0, n1):
                En, Bn = sim.E.clone(), sim.B.clone()
                sim.step(1)
                saved.append((En, Bn, sim.J.clone()))
            for En, Bn, Jn in reversed(saved):
                pic_adjoint_step(sim.h, En.data_ptr(), Bn.data_ptr(), Jn.data_ptr(), aE.data_ptr(), aB.data_ptr(),
                                 grad.data_ptr(), stream)
        torch.cuda.synchronize(self.device)
        g = grad.cpu().numpy()
        sim.close()
        return L, g


class StencilLossFn(torch.autograd.Function):
    """torch.autograd wrapper: loss = StencilLossFn.apply(C, problem) with C a CPU float64 tensor."""

    @staticmethod
    def forward(ctx, C, problem):
        L, g = problem.loss_and_grad(C.detach().cpu().numpy())
        ctx.save_for_backward(torch.from_numpy(g))
        return torch.tensor(L, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gL):
        (g,) = ctx.saved_tensors
        return gL * g, None
