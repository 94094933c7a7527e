"""PyTorch plumbing around the C ABI: device tensors for fields and particles, the caller's
CUDA stream, and host copies for inspection.  No PIC arithmetic happens here."""
import ctypes

import numpy as np
import torch

from . import (PIC_SOLVER_CUSTOM, PIC_SOLVER_YEE, encode_cells, pic_batch_create, pic_batch_destroy,
               pic_batch_instance, pic_batch_step, pic_bind_fields, pic_bind_species,
               pic_config, pic_create, pic_deposit, pic_destroy, pic_diag, pic_field_advance,
               pic_gather_push, pic_gauss, pic_get_coefficients, pic_get_count, pic_get_state, pic_rho,
               pic_sort, pic_step, pic_sync)


def make_config(ndim, nz, nx, ny=1, dz=1.0, dx=1.0, dy=1.0, dt=0.5, solver="yee", M=16, coef=None,
                fit_wk=0.0, fit_n=0.0, shape=1, moving_window=False, inject_species=-1,
                inject_ppc=(1, 1, 1), rho_bg=0.0, sort_every=0):
    c = pic_config()
    c.ndim, c.nz, c.nx, c.ny = int(ndim), int(nz), int(nx), int(ny if ndim == 3 else 1)
    c.dz, c.dx, c.dy, c.dt = float(dz), float(dx), float(dy), float(dt)
    c.solver = PIC_SOLVER_CUSTOM if solver == "custom" else PIC_SOLVER_YEE
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
