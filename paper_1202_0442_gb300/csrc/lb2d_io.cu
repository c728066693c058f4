// lb2d_io.cu -- input-data and restart text files: the read_data and
// write_restart commands (Sec. Commands).
//
// A fluid file holds nine sections, each a line with the section's name
// followed by its data lines:
//   relaxation_time  tau [alpha]      (alpha: two components only)
//   domain           Nx Ny            (sites 0..Nx x 0..Ny)
//   processors       px py
//   inlet / outlet   wall x0 x1 label style arguments   (one line per opening)
//   boundary         periodic | noslip | slip | mixed R | hybrid
//   field            force e<k> value ...; acceleration e<k> value ...;
//                    interforce G psi0 rho0; adhesiveforce G psi0 rho0
//   density          x y rho style    (rho = -11 marks a solid site)
//   momentum         x y f0 ... f8
// with the order rules of the command: domain before processors, field
// after relaxation_time, processors before density and momentum, boundary
// before density.  A solute file holds relaxation_time (tau_s), inlet /
// outlet (wall x0 x1 label style arguments), reaction (surface kr Cs style
// bmax), field (intersolute G psi0 C0), concentration (x y C [b]) and
// solute_modes (x y g_1 ... g_q); reaction precedes concentration.  Two
// components are written as <file>.fluid1 / <file>.fluid2, the solute as
// <file>.solute.
//
// Readings where the command leaves room (the same as the oracle's
// reader): every site is listed in density and, when present, in momentum;
// a mixed site may carry its R after the style word; the reaction line may
// carry b0 and the growth seed after bmax; D2Q9 solute lines carry g_0 ...
// g_8; a file without a momentum section, or read with "equilibrium",
// starts at the equilibrium of its densities and of the velocities its
// populations carry (zero without a momentum section).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "lbctx.h"

using namespace lbk;

namespace {

const char *const WALLS[4] = {"xlo", "xhi", "ylo", "yhi"};
const int EX9[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
const int EY9[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
constexpr double SOLID_RHO = -11.0;

const char *momentum_style(int st) {
  switch (st) {
    case OPEN_POISEUILLE: return "poiseuille";
    case OPEN_UNIFORM: return "uniform";
    case OPEN_DIRICHLET: return "dirichlet";
    case OPEN_GRADIENT: return "gradient";
    default: return nullptr;
  }
}

const char *solute_style(int st) {
  switch (st) {
    case SOL_DIRICHLET: return "dirichlet";
    case SOL_ADIABATIC: return "adiabatic";
    case SOL_FLUX: return "flux";
    default: return nullptr;
  }
}

// ------------------------------------------------------------- writing

// buffered text output with %.17g numbers (every FP64 value read back
// exactly)
struct Text {
  FILE *f = nullptr;
  std::vector<char> buf;
  explicit Text(const std::string &name) : f(fopen(name.c_str(), "w")), buf(1 << 20) {
    if (f) setvbuf(f, buf.data(), _IOFBF, buf.size());
  }
  ~Text() {
    if (f) fclose(f);
  }
  void num(double v) { fprintf(f, " %.17g", v); }
  bool close() {
    const bool ok = f && !ferror(f) && fclose(f) == 0;
    f = nullptr;
    return ok;
  }
};

void write_openings(Text &o, const lb_ctx *ctx, int kind, int comp, bool solute) {
  bool head = false;
  for (const Opening &op : ctx->open) {
    if (op.kind != kind) continue;
    if (solute && !solute_style(op.sstyle)) continue;
    if (!head) {
      fprintf(o.f, "%s\n", kind ? "outlet" : "inlet");
      head = true;
    }
    const std::string &label = op.label[solute ? 0 : comp];
    fprintf(o.f, "%s %d %d %s", WALLS[op.wall], op.a0, op.a1, label.c_str());
    if (solute) {
      fprintf(o.f, " %s", solute_style(op.sstyle));
      if (op.sstyle == SOL_FLUX) {
        o.num(op.sv);
        o.num(op.C);
      } else {
        o.num(op.C);
      }
    } else if (const char *st = momentum_style(op.style[comp])) {
      fprintf(o.f, " %s", st);
      if (op.style[comp] == OPEN_POISEUILLE || op.style[comp] == OPEN_UNIFORM) o.num(op.v[comp]);
      o.num(op.rho[comp]);
    }
    fprintf(o.f, "\n");
  }
  if (head) fprintf(o.f, "\n");
}

// the style word of solid site n for component c
std::string site_style(const lb_ctx *ctx, int c, size_t n) {
  char b[64];
  switch (ctx->bstyle) {
    case 1: return "slip";
    case 2: return "mixed";
    case 3: {
      const double R = ctx->solid[n] ? ctx->Rh[c][n] : 0.0;
      if (R == 0.0) return "noslip";
      if (R == 1.0) return "slip";
      snprintf(b, sizeof b, "mixed %.9g", R);
      return b;
    }
    default: return "noslip";
  }
}

int write_fluid(lb_ctx *ctx, int c, const std::string &name, const std::vector<uint8_t> &mask) {
  const int nx = ctx->nx, ny = ctx->ny;
  const size_t nn = (size_t)nx * ny;
  std::vector<double> f(9 * nn);
  TRY(lb_get_populations(ctx, c + 1, f.data()));
  Text o(name);
  if (!o.f) return ctx->fail(LB_E_ARG, "cannot write '%s'", name.c_str());
  fprintf(o.f, "relaxation_time\n");
  o.num(ctx->tau[c]);
  if (ctx->nc == 2) o.num(ctx->alpha[c]);  // the density-ratio parameter of multicomponent runs
  fprintf(o.f, "\n\ndomain\n%d %d\n\nprocessors\n%d %d\n\n", nx - 1, ny - 1, ctx->px, ctx->py);
  write_openings(o, ctx, 0, c, false);
  write_openings(o, ctx, 1, c, false);
  fprintf(o.f, "boundary\n");
  if (!ctx->have_style) fprintf(o.f, "periodic\n\n");
  else if (ctx->bstyle == 2) fprintf(o.f, "mixed %.17g\n\n", ctx->slipR);
  else fprintf(o.f, "%s\n\n", ctx->bstyle == 0 ? "noslip" : ctx->bstyle == 1 ? "slip" : "hybrid");
  fprintf(o.f, "field\nforce e1");
  o.num(ctx->fave[c][0]);
  fprintf(o.f, " e2");
  o.num(ctx->fave[c][1]);
  fprintf(o.f, "\nacceleration e1");
  o.num(ctx->acc[c][0]);
  fprintf(o.f, " e2");
  o.num(ctx->acc[c][1]);
  fprintf(o.f, "\n");
  if (ctx->sc) {
    fprintf(o.f, "interforce");
    o.num(ctx->G);
    o.num(ctx->psi0);
    o.num(ctx->sc_rho0);
    fprintf(o.f, "\n");
  }
  if (ctx->ads[c]) {
    fprintf(o.f, "adhesiveforce");
    o.num(ctx->Gads[c]);
    o.num(ctx->ads_psi0[c]);
    o.num(ctx->ads_rho0[c]);
    fprintf(o.f, "\n");
  }
  fprintf(o.f, "\ndensity\n");
  for (int y = 0; y < ny; y++)
    for (int x = 0; x < nx; x++) {
      const size_t n = (size_t)y * nx + x;
      double rho = SOLID_RHO;
      if (!mask[n]) {
        rho = 0.0;
        for (int i = 0; i < 9; i++) rho += f[i * nn + n];
      }
      fprintf(o.f, "%d %d", x, y);
      o.num(rho);
      fprintf(o.f, " %s\n", site_style(ctx, c, n).c_str());
    }
  fprintf(o.f, "\nmomentum\n");
  for (int y = 0; y < ny; y++)
    for (int x = 0; x < nx; x++) {
      const size_t n = (size_t)y * nx + x;
      fprintf(o.f, "%d %d", x, y);
      for (int i = 0; i < 9; i++) o.num(mask[n] ? 0.0 : f[i * nn + n]);
      fprintf(o.f, "\n");
    }
  if (!o.close()) return ctx->fail(LB_E_ARG, "writing '%s' failed", name.c_str());
  return LB_OK;
}

int write_solute(lb_ctx *ctx, const std::string &name, const std::vector<uint8_t> &mask) {
  const int nx = ctx->nx, ny = ctx->ny, q = ctx->qs;
  const size_t nn = (size_t)nx * ny;
  std::vector<double> g((size_t)q * nn), b(nn);
  TRY(lb_get_solute(ctx, g.data(), nullptr, b.data()));
  Text o(name);
  if (!o.f) return ctx->fail(LB_E_ARG, "cannot write '%s'", name.c_str());
  fprintf(o.f, "relaxation_time\n");
  o.num(ctx->taus);
  fprintf(o.f, "\n\n");
  write_openings(o, ctx, 0, 0, true);
  write_openings(o, ctx, 1, 0, true);
  if (ctx->react) {
    fprintf(o.f, "reaction\nsurface");
    o.num(ctx->kr);
    o.num(ctx->Cs);
    fprintf(o.f, " growth");
    o.num(ctx->bmax);
    o.num(ctx->b0);
    fprintf(o.f, " %llu\n\n", (unsigned long long)ctx->seed);
  }
  if (ctx->inter) {
    fprintf(o.f, "field\nintersolute");
    o.num(ctx->isG);
    o.num(ctx->ispsi0);
    o.num(ctx->isC0);
    fprintf(o.f, "\n\n");
  }
  fprintf(o.f, "concentration\n");
  for (int y = 0; y < ny; y++)
    for (int x = 0; x < nx; x++) {
      const size_t n = (size_t)y * nx + x;
      double C = 0.0;
      if (!mask[n])
        for (int i = 0; i < q; i++) C += g[i * nn + n];
      fprintf(o.f, "%d %d", x, y);
      o.num(C);
      if (ctx->react) o.num(b[n]);
      fprintf(o.f, "\n");
    }
  fprintf(o.f, "\nsolute_modes\n");
  for (int y = 0; y < ny; y++)
    for (int x = 0; x < nx; x++) {
      const size_t n = (size_t)y * nx + x;
      fprintf(o.f, "%d %d", x, y);
      for (int i = 0; i < q; i++) o.num(mask[n] ? 0.0 : g[i * nn + n]);
      fprintf(o.f, "\n");
    }
  if (!o.close()) return ctx->fail(LB_E_ARG, "writing '%s' failed", name.c_str());
  return LB_OK;
}

// ------------------------------------------------------------- reading

struct Line {
  int no = 0;
  std::vector<const char *> tok;
};

struct Section {
  std::string name;
  int no = 0, order = 0;
  std::vector<Line> lines;
};

// a file split into sections; the text is kept and tokenised in place
struct DataFile {
  std::string name, text;
  std::vector<Section> sec;

  const Section *find(const char *s) const {
    for (const Section &x : sec)
      if (x.name == s) return &x;
    return nullptr;
  }
  int order(const char *s) const {
    const Section *x = find(s);
    return x ? x->order : -1;
  }
};

int load(lb_ctx *ctx, const std::string &name, const char *const *names, int nnames, DataFile &d) {
  d.name = name;
  FILE *f = fopen(name.c_str(), "rb");
  if (!f) return ctx->fail(LB_E_ARG, "cannot read '%s'", name.c_str());
  char chunk[1 << 16];
  size_t k;
  while ((k = fread(chunk, 1, sizeof chunk, f)) > 0) d.text.append(chunk, k);
  fclose(f);
  d.text.push_back('\0');
  char *p = &d.text[0];
  int no = 0;
  while (*p) {
    no++;
    char *eol = strchr(p, '\n');
    char *next = eol ? eol + 1 : p + strlen(p);
    if (eol) *eol = '\0';
    Line ln;
    ln.no = no;
    char *save = nullptr;
    for (char *t = strtok_r(p, " \t\r", &save); t; t = strtok_r(nullptr, " \t\r", &save)) ln.tok.push_back(t);
    p = next;
    if (ln.tok.empty()) continue;
    bool head = false;
    if (ln.tok.size() == 1)
      for (int i = 0; i < nnames; i++)
        if (!strcmp(ln.tok[0], names[i])) head = true;
    if (head) {
      if (d.find(ln.tok[0])) return ctx->fail(LB_E_ARG, "%s:%d: section '%s' repeated", name.c_str(), no, ln.tok[0]);
      Section s;
      s.name = ln.tok[0];
      s.no = no;
      s.order = (int)d.sec.size();
      d.sec.push_back(std::move(s));
      continue;
    }
    if (d.sec.empty()) return ctx->fail(LB_E_ARG, "%s:%d: data before the first section", name.c_str(), no);
    d.sec.back().lines.push_back(std::move(ln));
  }
  return LB_OK;
}

bool to_double(const char *s, double &v) {
  char *end;
  v = strtod(s, &end);
  return end != s && *end == '\0' && std::isfinite(v);
}

bool to_int(const char *s, int &v) {
  char *end;
  long x = strtol(s, &end, 10);
  if (end == s || *end != '\0' || x < INT32_MIN || x > INT32_MAX) return false;
  v = (int)x;
  return true;
}

// numbers t[k0..k0+n) of line ln into out
int numbers(lb_ctx *ctx, const DataFile &d, const Line &ln, size_t k0, size_t n, double *out) {
  if (ln.tok.size() < k0 + n)
    return ctx->fail(LB_E_ARG, "%s:%d: %zu values expected", d.name.c_str(), ln.no, k0 + n);
  for (size_t k = 0; k < n; k++)
    if (!to_double(ln.tok[k0 + k], out[k]))
      return ctx->fail(LB_E_ARG, "%s:%d: '%s' is not a number", d.name.c_str(), ln.no, ln.tok[k0 + k]);
  return LB_OK;
}

// site (x, y) at the start of a line -> node index
int site(lb_ctx *ctx, const DataFile &d, const Line &ln, int nx, int ny, size_t &n) {
  int x, y;
  if (ln.tok.size() < 2 || !to_int(ln.tok[0], x) || !to_int(ln.tok[1], y))
    return ctx->fail(LB_E_ARG, "%s:%d: a site 'x y' expected", d.name.c_str(), ln.no);
  if (x < 0 || x >= nx || y < 0 || y >= ny)
    return ctx->fail(LB_E_ARG, "%s:%d: site (%d,%d) outside the %d x %d lattice", d.name.c_str(), ln.no, x, y, nx, ny);
  n = (size_t)y * nx + x;
  return LB_OK;
}

// an opening line of either file kind
struct OpenLine {
  int kind = 0, wall = 0, a0 = 0, a1 = 0, no = 0;
  std::string label, style;
  std::vector<double> args;
};

int openings(lb_ctx *ctx, const DataFile &d, std::vector<OpenLine> &out) {
  for (int kind = 0; kind < 2; kind++) {
    const Section *s = d.find(kind ? "outlet" : "inlet");
    if (!s) continue;
    for (const Line &ln : s->lines) {
      OpenLine o;
      o.kind = kind;
      o.no = ln.no;
      o.wall = -1;
      if (ln.tok.size() < 4) return ctx->fail(LB_E_ARG, "%s:%d: 'wall x0 x1 label ...' expected", d.name.c_str(), ln.no);
      for (int w = 0; w < 4; w++)
        if (!strcmp(ln.tok[0], WALLS[w])) o.wall = w;
      if (o.wall < 0 || !to_int(ln.tok[1], o.a0) || !to_int(ln.tok[2], o.a1))
        return ctx->fail(LB_E_ARG, "%s:%d: 'wall x0 x1 label ...' expected", d.name.c_str(), ln.no);
      o.label = ln.tok[3];
      if (ln.tok.size() > 4) {
        o.style = ln.tok[4];
        o.args.resize(ln.tok.size() - 5);
        TRY(numbers(ctx, d, ln, 5, o.args.size(), o.args.data()));
      }
      out.push_back(o);
    }
  }
  return LB_OK;
}

// one fluid component's file
struct FluidData {
  DataFile d;
  double tau = 0, alpha = -1;
  int Nx = -1, Ny = -1, px = 0, py = 0;
  std::vector<OpenLine> open;
  std::string bstyle;
  double bR = 0;
  std::vector<std::pair<int, double>> force, accel;
  bool inter = false, ads = false;
  double iG = 0, ipsi0 = 0, irho0 = 0, aG = 0, apsi0 = 0, arho0 = 0;
  std::vector<double> rho, f, R;  // density, populations, per-site R
  std::vector<uint8_t> solid;
  bool has_density = false, has_f = false;
};

const char *const FLUID_SECTIONS[9] = {"relaxation_time", "domain", "processors", "inlet", "outlet",
                                       "boundary", "field", "density", "momentum"};
const char *const SOLUTE_SECTIONS[7] = {"relaxation_time", "inlet", "outlet", "reaction", "field",
                                        "concentration", "solute_modes"};

// "e<k>" -> k
bool mode_of(const char *s, int &k) { return s[0] == 'e' && to_int(s + 1, k) && k >= 0 && k <= 8; }

int parse_fluid(lb_ctx *ctx, const std::string &name, FluidData &F) {
  DataFile &d = F.d;
  TRY(load(ctx, name, FLUID_SECTIONS, 9, d));
  const char *nm = name.c_str();
  auto before = [&](const char *a, const char *b) {
    return d.order(a) < 0 || d.order(b) < 0 || d.order(a) < d.order(b);
  };
  if (d.order("processors") >= 0 && d.order("domain") >= 0 && !before("domain", "processors"))
    return ctx->fail(LB_E_ARG, "%s: the section domain must precede processors", nm);
  if (d.order("field") >= 0 && !(d.order("relaxation_time") >= 0 && before("relaxation_time", "field")))
    return ctx->fail(LB_E_ARG, "%s: the section field must follow relaxation_time", nm);
  if (!before("processors", "density") || !before("processors", "momentum"))
    return ctx->fail(LB_E_ARG, "%s: the section processors must precede density and momentum", nm);
  if (!before("boundary", "density")) return ctx->fail(LB_E_ARG, "%s: the section boundary must precede density", nm);
  auto one_line = [&](const Section *s) -> const Line * {
    return (s && !s->lines.empty()) ? &s->lines[0] : nullptr;
  };
  if (const Line *ln = one_line(d.find("relaxation_time"))) {
    double v[2] = {0, -1};
    TRY(numbers(ctx, d, *ln, 0, ln->tok.size() >= 2 ? 2 : 1, v));
    F.tau = v[0];
    F.alpha = v[1];
  }
  if (const Line *ln = one_line(d.find("domain"))) {
    if (ln->tok.size() != 2 || !to_int(ln->tok[0], F.Nx) || !to_int(ln->tok[1], F.Ny) || F.Nx < 0 || F.Ny < 0)
      return ctx->fail(LB_E_ARG, "%s:%d: 'Nx Ny' expected", nm, ln->no);
  }
  if (const Line *ln = one_line(d.find("processors"))) {
    if (ln->tok.size() != 2 || !to_int(ln->tok[0], F.px) || !to_int(ln->tok[1], F.py))
      return ctx->fail(LB_E_ARG, "%s:%d: 'px py' expected", nm, ln->no);
  }
  TRY(openings(ctx, d, F.open));
  if (const Line *ln = one_line(d.find("boundary"))) {
    F.bstyle = ln->tok[0];
    if (F.bstyle == "mixed") {
      if (ln->tok.size() < 2 || !to_double(ln->tok[1], F.bR))
        return ctx->fail(LB_E_ARG, "%s:%d: mixed needs its reflection coefficient", nm, ln->no);
    } else if (F.bstyle != "periodic" && F.bstyle != "noslip" && F.bstyle != "slip" && F.bstyle != "hybrid") {
      return ctx->fail(LB_E_ARG, "%s:%d: unknown boundary style '%s'", nm, ln->no, ln->tok[0]);
    }
  }
  if (const Section *s = d.find("field")) {
    for (const Line &ln : s->lines) {
      const std::string key = ln.tok[0];
      if (key == "force" || key == "acceleration") {
        if (ln.tok.size() % 2 != 1) return ctx->fail(LB_E_ARG, "%s:%d: 'mode value' pairs expected", nm, ln.no);
        for (size_t k = 1; k + 1 < ln.tok.size(); k += 2) {
          int m;
          double v;
          if (!mode_of(ln.tok[k], m) || !to_double(ln.tok[k + 1], v))
            return ctx->fail(LB_E_ARG, "%s:%d: 'e<k> value' expected", nm, ln.no);
          (key == "force" ? F.force : F.accel).push_back({m, v});
        }
      } else if (key == "interforce" || key == "adhesiveforce") {
        double v[3];
        TRY(numbers(ctx, d, ln, 1, 3, v));
        if (key == "interforce") {
          F.inter = true;
          F.iG = v[0], F.ipsi0 = v[1], F.irho0 = v[2];
        } else {
          F.ads = true;
          F.aG = v[0], F.apsi0 = v[1], F.arho0 = v[2];
        }
      } else {
        return ctx->fail(LB_E_ARG, "%s:%d: unknown field item '%s'", nm, ln.no, ln.tok[0]);
      }
    }
  }
  return LB_OK;
}

// the density and momentum sections of a fluid file on an nx x ny lattice
int parse_sites(lb_ctx *ctx, FluidData &F, int nx, int ny, double mixedR) {
  const DataFile &d = F.d;
  const size_t nn = (size_t)nx * ny;
  if (const Section *s = d.find("density")) {
    F.has_density = true;
    F.rho.assign(nn, 0.0);
    F.solid.assign(nn, 0);
    F.R.assign(nn, 0.0);
    std::vector<uint8_t> seen(nn, 0);
    for (const Line &ln : s->lines) {
      size_t n;
      TRY(site(ctx, d, ln, nx, ny, n));
      TRY(numbers(ctx, d, ln, 2, 1, &F.rho[n]));
      seen[n] = 1;
      F.solid[n] = F.rho[n] == SOLID_RHO;
      if (ln.tok.size() > 3) {
        const std::string st = ln.tok[3];
        if (st == "slip") F.R[n] = 1.0;
        else if (st == "mixed") {
          F.R[n] = mixedR;
          if (ln.tok.size() > 4) TRY(numbers(ctx, d, ln, 4, 1, &F.R[n]));
        } else if (st != "noslip") {
          return ctx->fail(LB_E_ARG, "%s:%d: unknown site style '%s'", d.name.c_str(), ln.no, ln.tok[3]);
        }
      }
      if (!F.solid[n] && !(F.rho[n] > 0))
        return ctx->fail(LB_E_ARG, "%s:%d: density must be positive (or -11 for a solid site)", d.name.c_str(), ln.no);
    }
    if (std::count(seen.begin(), seen.end(), 1) != (long)nn)
      return ctx->fail(LB_E_ARG, "%s: the section density lists %ld of the %zu sites", d.name.c_str(),
                       (long)std::count(seen.begin(), seen.end(), 1), nn);
  }
  if (const Section *s = d.find("momentum")) {
    F.has_f = true;
    F.f.assign(9 * nn, 0.0);
    std::vector<uint8_t> seen(nn, 0);
    for (const Line &ln : s->lines) {
      size_t n;
      TRY(site(ctx, d, ln, nx, ny, n));
      double v[9];
      TRY(numbers(ctx, d, ln, 2, 9, v));
      for (int i = 0; i < 9; i++) F.f[i * nn + n] = v[i];
      seen[n] = 1;
    }
    if (std::count(seen.begin(), seen.end(), 1) != (long)nn)
      return ctx->fail(LB_E_ARG, "%s: the section momentum lists %ld of the %zu sites", d.name.c_str(),
                       (long)std::count(seen.begin(), seen.end(), 1), nn);
  }
  if (!F.has_density && !F.has_f)
    return ctx->fail(LB_E_ARG, "%s: neither a density nor a momentum section", d.name.c_str());
  return LB_OK;
}

struct SoluteData {
  DataFile d;
  double taus = 0;
  int q = 0;
  std::vector<OpenLine> open;
  bool react = false, inter = false, has_b = false, has_C = false, has_g = false;
  double kr = 0, Cs = 0, bmax = 0, b0 = 0, iG = 0, ipsi0 = 0, iC0 = 0;
  unsigned long long seed = 0;
  bool has_b0 = false, has_seed = false;
  std::string rstyle;
  std::vector<double> C, b, g;
};

int parse_solute(lb_ctx *ctx, const std::string &name, int nx, int ny, SoluteData &S) {
  DataFile &d = S.d;
  TRY(load(ctx, name, SOLUTE_SECTIONS, 7, d));
  const char *nm = name.c_str();
  if (d.order("field") >= 0 && !(d.order("relaxation_time") >= 0 && d.order("relaxation_time") < d.order("field")))
    return ctx->fail(LB_E_ARG, "%s: the section field must follow relaxation_time", nm);
  if (d.order("reaction") >= 0 && d.order("concentration") >= 0 && d.order("reaction") > d.order("concentration"))
    return ctx->fail(LB_E_ARG, "%s: the section reaction must precede concentration", nm);
  if (const Section *s = d.find("relaxation_time"))
    if (!s->lines.empty()) TRY(numbers(ctx, d, s->lines[0], 0, 1, &S.taus));
  TRY(openings(ctx, d, S.open));
  if (const Section *s = d.find("reaction")) {
    for (const Line &ln : s->lines) {
      if (strcmp(ln.tok[0], "surface") || ln.tok.size() < 5)
        return ctx->fail(LB_E_ARG, "%s:%d: 'surface kr Cs style bmax' expected", nm, ln.no);
      S.react = true;
      double v[2] = {0, 0};
      TRY(numbers(ctx, d, ln, 1, 2, v));
      S.kr = v[0];
      S.Cs = v[1];
      S.rstyle = ln.tok[3];
      TRY(numbers(ctx, d, ln, 4, 1, &S.bmax));
      if (ln.tok.size() > 5) {
        TRY(numbers(ctx, d, ln, 5, 1, &S.b0));
        S.has_b0 = true;
      }
      if (ln.tok.size() > 6) {
        char *end;
        S.seed = strtoull(ln.tok[6], &end, 10);
        if (*end) return ctx->fail(LB_E_ARG, "%s:%d: the growth seed must be an integer", nm, ln.no);
        S.has_seed = true;
      }
    }
  }
  if (const Section *s = d.find("field")) {
    for (const Line &ln : s->lines) {
      if (strcmp(ln.tok[0], "intersolute")) return ctx->fail(LB_E_ARG, "%s:%d: unknown field item '%s'", nm, ln.no, ln.tok[0]);
      double v[3];
      TRY(numbers(ctx, d, ln, 1, 3, v));
      S.inter = true;
      S.iG = v[0], S.ipsi0 = v[1], S.iC0 = v[2];
    }
  }
  const size_t nn = (size_t)nx * ny;
  if (const Section *s = d.find("concentration")) {
    S.has_C = true;
    S.C.assign(nn, 0.0);
    S.b.assign(nn, 0.0);
    std::vector<uint8_t> seen(nn, 0);
    for (const Line &ln : s->lines) {
      size_t n;
      TRY(site(ctx, d, ln, nx, ny, n));
      TRY(numbers(ctx, d, ln, 2, 1, &S.C[n]));
      if (ln.tok.size() > 3) {
        TRY(numbers(ctx, d, ln, 3, 1, &S.b[n]));
        S.has_b = true;
      }
      seen[n] = 1;
    }
    if (std::count(seen.begin(), seen.end(), 1) != (long)nn)
      return ctx->fail(LB_E_ARG, "%s: the section concentration lists %ld of the %zu sites", nm,
                       (long)std::count(seen.begin(), seen.end(), 1), nn);
  }
  if (const Section *s = d.find("solute_modes")) {
    S.has_g = true;
    std::vector<uint8_t> seen(nn, 0);
    for (const Line &ln : s->lines) {
      size_t n;
      TRY(site(ctx, d, ln, nx, ny, n));
      const int q = (int)ln.tok.size() - 2;
      if (q != 4 && q != 9)
        return ctx->fail(LB_E_ARG, "%s:%d: 4 (D2Q4) or 9 (D2Q9) solute modes expected", nm, ln.no);
      if (!S.q) {
        S.q = q;
        S.g.assign((size_t)q * nn, 0.0);
      }
      if (q != S.q) return ctx->fail(LB_E_ARG, "%s:%d: %d modes after lines of %d", nm, ln.no, q, S.q);
      double v[9];
      TRY(numbers(ctx, d, ln, 2, q, v));
      for (int i = 0; i < q; i++) S.g[i * nn + n] = v[i];
      seen[n] = 1;
    }
    if (std::count(seen.begin(), seen.end(), 1) != (long)nn)
      return ctx->fail(LB_E_ARG, "%s: the section solute_modes lists %ld of the %zu sites", nm,
                       (long)std::count(seen.begin(), seen.end(), 1), nn);
  }
  if (!S.has_C && !S.has_g) return ctx->fail(LB_E_ARG, "%s: neither a concentration nor a solute_modes section", nm);
  return LB_OK;
}

int find_opening(lb_ctx *ctx, const OpenLine &o) {
  for (size_t k = 0; k < ctx->open.size(); k++) {
    const Opening &p = ctx->open[k];
    if (p.kind == o.kind && p.wall == o.wall && p.a0 == o.a0 && p.a1 == o.a1) return (int)k;
  }
  return -1;
}

int apply_momentum_style(lb_ctx *ctx, const DataFile &d, const OpenLine &o) {
  if (o.style.empty()) return LB_OK;
  double v = 0, rho = 0;
  if (o.style == "poiseuille" || o.style == "uniform") {
    if (o.args.size() < 2) return ctx->fail(LB_E_ARG, "%s:%d: '%s' needs a velocity and a density", d.name.c_str(), o.no, o.style.c_str());
    v = o.args[0];
    rho = o.args[1];
  } else {
    if (o.args.empty()) return ctx->fail(LB_E_ARG, "%s:%d: '%s' needs a density", d.name.c_str(), o.no, o.style.c_str());
    rho = o.args[0];
  }
  return o.kind ? lb_outlet_momentum(ctx, o.label.c_str(), o.style.c_str(), v, rho)
                : lb_inlet_momentum(ctx, o.label.c_str(), o.style.c_str(), v, rho);
}

}  // namespace

int write_data_files(lb_ctx *ctx, const std::string &base) {
  NvtxRange range("write_restart");
  if (ctx->rank >= 0) return ctx->fail(LB_E_UNSUPPORTED, "a slab writes no input-data file: gather the lattice first");
  if (!ctx->committed) return ctx->fail(LB_E_ORDER, "no device state yet");
  std::vector<uint8_t> mask((size_t)ctx->nx * ctx->ny);
  TRY(lb_get_mask(ctx, mask.data()));
  if (ctx->nc == 1) TRY(write_fluid(ctx, 0, base, mask));
  else
    for (int c = 0; c < 2; c++) TRY(write_fluid(ctx, c, base + ".fluid" + std::to_string(c + 1), mask));
  if (ctx->qs) TRY(write_solute(ctx, base + ".solute", mask));
  return LB_OK;
}

extern "C" {

int lb_lattice_info(lb_ctx *ctx, int *nx, int *ny, int *ncomp, int *q, int *px, int *py) {
  NEED_CTX();
  if (!ctx->have_lattice) return ctx->fail(LB_E_ORDER, "no lattice yet");
  if (nx) *nx = ctx->nx;
  if (ny) *ny = ctx->ny;
  if (ncomp) *ncomp = ctx->nc;
  if (q) *q = ctx->qs;
  if (px) *px = ctx->px;
  if (py) *py = ctx->py;
  return LB_OK;
}

int lb_write_data(lb_ctx *ctx, const char *file) {
  NEED_CTX();
  if (!file || !*file) return ctx->fail(LB_E_ARG, "no file name");
  return write_data_files(ctx, file);
}

int lb_write_restart(lb_ctx *ctx, const char *file, int Nf) {
  NEED_CTX();
  if (Nf < 0) return ctx->fail(LB_E_ARG, "Nf must be >= 0");
  if (Nf > 0 && (!file || !*file)) return ctx->fail(LB_E_ARG, "no file name");
  if (Nf > 0 && ctx->rank >= 0) return ctx->fail(LB_E_UNSUPPORTED, "a slab writes no restart file");
  if (Nf > 0 && ctx->iterated)
    return ctx->fail(LB_E_ORDER, "write_restart must precede the iteration command (lb_write_data writes now)");
  ctx->restart_nf = Nf;
  ctx->restart_file = Nf > 0 ? file : "";
  return LB_OK;
}

int lb_read_data(lb_ctx *ctx, const char *file, const char *args) {
  NEED_CTX();
  NvtxRange range("read_data");
  if (!file || !*file) return ctx->fail(LB_E_ARG, "no file name");
  if (ctx->committed) return ctx->fail(LB_E_ORDER, "read_data must precede the first iteration");
  if (ctx->rank >= 0) return ctx->fail(LB_E_UNSUPPORTED, "read_data into a slab is not built");
  bool fluids = false, solute = false, equilibrium = false;
  if (args) {
    std::string a(args);
    for (char &ch : a)
      if (ch == ',') ch = ' ';
    std::vector<char> buf(a.begin(), a.end());
    buf.push_back('\0');
    char *save = nullptr;
    for (char *t = strtok_r(buf.data(), " \t", &save); t; t = strtok_r(nullptr, " \t", &save)) {
      if (!strcmp(t, "fluids")) fluids = true;
      else if (!strcmp(t, "solute")) solute = true;
      else if (!strcmp(t, "equilibrium")) equilibrium = true;
      else return ctx->fail(LB_E_ARG, "read_data arguments are fluids, solute and equilibrium, not '%s'", t);
    }
  }
  const int nfl = fluids ? 2 : 1;
  std::vector<FluidData> F(nfl);
  for (int c = 0; c < nfl; c++)
    TRY(parse_fluid(ctx, fluids ? std::string(file) + ".fluid" + std::to_string(c + 1) : std::string(file), F[c]));
  // domain, relaxation times, processors
  int Nx = F[0].Nx, Ny = F[0].Ny;
  for (int c = 1; c < nfl; c++)
    if (F[c].Nx != Nx || F[c].Ny != Ny) return ctx->fail(LB_E_ARG, "the two fluid files give different domains");
  if (Nx < 0 && !ctx->have_lattice) return ctx->fail(LB_E_ORDER, "no domain section and no lattice command");
  const double tau0 = F[0].tau > 0 ? F[0].tau : ctx->tau[0];
  if (Nx >= 0 && (!ctx->have_lattice || ctx->nx != Nx + 1 || ctx->ny != Ny + 1))
    TRY(lb_lattice(ctx, "d2q9", Nx + 1, Ny + 1, tau0));
  const int nx = ctx->nx, ny = ctx->ny;
  const size_t nn = (size_t)nx * ny;
  if (nfl == 2) {
    double t[2], al[2];
    for (int c = 0; c < 2; c++) {
      t[c] = F[c].tau > 0 ? F[c].tau : ctx->tau[c];
      al[c] = F[c].alpha >= 0 ? F[c].alpha : ctx->alpha[c];
    }
    TRY(lb_fluids(ctx, t[0], t[1], al[0], al[1]));
  } else {
    if (ctx->nc != 1) return ctx->fail(LB_E_ARG, "two fluids are read with the argument fluids");
    if (!(tau0 > 0.5)) return ctx->fail(LB_E_ARG, "tau must exceed 1/2");
    ctx->tau[0] = ctx->tau[1] = tau0;
    // a density-ratio parameter belongs to multicomponent runs only: a
    // single component keeps the weights of Eq. (2)
  }
  if (F[0].px > 0) TRY(lb_processors(ctx, F[0].px, F[0].py));
  // boundary style and the solid sites (the file's sites replace the mask)
  const std::string &bs = F[0].bstyle;
  for (int c = 0; c < nfl; c++) TRY(parse_sites(ctx, F[c], nx, ny, F[0].bR));
  if (!bs.empty() && bs != "periodic") TRY(lb_boundary_style(ctx, bs.c_str(), F[0].bR));
  if (F[0].has_density) {
    for (int c = 1; c < nfl; c++)
      if (F[c].has_density && F[c].solid != F[0].solid)
        return ctx->fail(LB_E_ARG, "the two fluid files mark different solid sites");
    if (std::count(F[0].solid.begin(), F[0].solid.end(), 1) && !ctx->have_style)
      TRY(lb_boundary_style(ctx, "noslip", 0.0));
    ctx->solid = F[0].solid;
    if (ctx->bstyle == 3)
      for (int c = 0; c < 2; c++)
        for (size_t n = 0; n < nn; n++)
          ctx->Rh[c][n] = ctx->solid[n] ? (float)F[std::min(c, nfl - 1)].R[n] : 0.0f;
  }
  // openings: one line per opening in each fluid file, matched by place
  for (size_t k = 0; k < F[0].open.size(); k++) {
    const OpenLine &o = F[0].open[k];
    const OpenLine *o2 = nullptr;
    if (nfl == 2) {
      for (const OpenLine &p : F[1].open)
        if (p.kind == o.kind && p.wall == o.wall && p.a0 == o.a0 && p.a1 == o.a1) o2 = &p;
      if (!o2) return ctx->fail(LB_E_ARG, "%s:%d: the opening has no line in the second fluid file", F[0].d.name.c_str(), o.no);
    }
    if (find_opening(ctx, o) < 0) {
      TRY(o.kind ? lb_outlet(ctx, WALLS[o.wall], o.a0, o.a1, o.label.c_str(), o2 ? o2->label.c_str() : nullptr)
                 : lb_inlet(ctx, WALLS[o.wall], o.a0, o.a1, o.label.c_str(), o2 ? o2->label.c_str() : nullptr));
    } else {
      Opening &p = ctx->open[find_opening(ctx, o)];
      p.label[0] = o.label;
      if (o2) p.label[1] = o2->label;
    }
    TRY(apply_momentum_style(ctx, F[0].d, o));
    if (o2) TRY(apply_momentum_style(ctx, F[1].d, *o2));
  }
  if (nfl == 2 && F[1].open.size() != F[0].open.size())
    return ctx->fail(LB_E_ARG, "the two fluid files list different openings");
  // fields
  for (int c = 0; c < nfl; c++) {
    for (auto &m : F[c].force) TRY(lb_aveforce(ctx, m.first, m.second, c + 1));
    for (auto &m : F[c].accel) TRY(lb_aveacceleration(ctx, m.first, m.second, c + 1));
    if (F[c].ads) TRY(lb_adhesiveforce(ctx, F[c].aG, F[c].apsi0, F[c].arho0, c + 1));
  }
  if (F[0].inter) TRY(lb_interforce(ctx, F[0].iG, F[0].ipsi0, F[0].irho0));
  // the state: populations, or the equilibrium of the densities and
  // velocities read
  std::vector<double> jx(nn, 0.0), jy(nn, 0.0), rs(nn, 0.0);  // solvent momentum and density
  for (int c = 0; c < nfl; c++) {
    FluidData &D = F[c];
    lb_ctx::ReadState r;
    if (D.has_f && !equilibrium) {
      r.kind = 1;
      r.a = D.f;
    } else {
      r.kind = 2;
      r.a.assign(nn, 0.0);
      r.ux.assign(nn, 0.0);
      r.uy.assign(nn, 0.0);
      for (size_t n = 0; n < nn; n++) {
        if (ctx->solid[n]) continue;
        double rho = 0, px = 0, py = 0;
        if (D.has_f)
          for (int i = 0; i < 9; i++) {
            rho += D.f[i * nn + n];
            px += EX9[i] * D.f[i * nn + n];
            py += EY9[i] * D.f[i * nn + n];
          }
        if (D.has_density) rho = D.rho[n];
        if (!(rho > 0)) return ctx->fail(LB_E_ARG, "%s: site (%zu,%zu) has no positive density", D.d.name.c_str(), n % nx, n / nx);
        r.a[n] = rho;
        r.ux[n] = px / rho;
        r.uy[n] = py / rho;
      }
    }
    for (size_t n = 0; n < nn; n++) {
      if (ctx->solid[n]) continue;
      if (r.kind == 1) {
        for (int i = 0; i < 9; i++) {
          rs[n] += r.a[i * nn + n];
          jx[n] += EX9[i] * r.a[i * nn + n];
          jy[n] += EY9[i] * r.a[i * nn + n];
        }
      } else {
        rs[n] += r.a[n];
        jx[n] += r.a[n] * r.ux[n];
        jy[n] += r.a[n] * r.uy[n];
      }
    }
    // the file's state replaces one painted before read_data
    ctx->painted_f[c] = false;
    ctx->paint_f[c].clear();
    ctx->paint_base[c].clear();
    ctx->rf[c] = std::move(r);
  }
  if (!solute) return LB_OK;
  SoluteData S;
  TRY(parse_solute(ctx, std::string(file) + ".solute", nx, ny, S));
  const int q = S.q ? S.q : (ctx->qs ? ctx->qs : 4);
  const double taus = S.taus > 0 ? S.taus : ctx->taus;
  TRY(lb_solute(ctx, taus, q));
  for (const OpenLine &o : S.open) {
    const int k = find_opening(ctx, o);
    if (k < 0) return ctx->fail(LB_E_ARG, "%s:%d: a solute opening needs the fluid opening at the same place", S.d.name.c_str(), o.no);
    double C = 0, v = 0;
    if (o.style == "flux") {
      if (o.args.size() < 2) return ctx->fail(LB_E_ARG, "%s:%d: flux needs a velocity and a concentration", S.d.name.c_str(), o.no);
      v = o.args[0];
      C = o.args[1];
    } else {
      if (o.args.empty()) return ctx->fail(LB_E_ARG, "%s:%d: '%s' needs a concentration", S.d.name.c_str(), o.no, o.style.c_str());
      C = o.args[0];
    }
    const std::string label = ctx->open[k].label[0];
    TRY(o.kind ? lb_outlet_solute(ctx, label.c_str(), o.style.c_str(), C, v)
               : lb_inlet_solute(ctx, label.c_str(), o.style.c_str(), C, v));
  }
  if (S.react)
    TRY(lb_surface_reaction(ctx, S.kr, S.Cs, S.rstyle.c_str(), S.has_b0 ? S.b0 : ctx->b0, S.bmax,
                            S.has_seed ? S.seed : ctx->seed));
  if (S.inter) TRY(lb_intersolute(ctx, S.iG, S.ipsi0, S.iC0));
  lb_ctx::ReadState r;
  if (S.has_g && !equilibrium) {
    r.kind = 1;
    r.a = S.g;
  } else {
    if (!S.has_C) {
      S.C.assign(nn, 0.0);
      for (size_t n = 0; n < nn; n++)
        for (int i = 0; i < q; i++) S.C[n] += S.g[i * nn + n];
    }
    r.kind = 2;
    r.a = S.C;
    r.ux.assign(nn, 0.0);
    r.uy.assign(nn, 0.0);
    for (size_t n = 0; n < nn; n++)
      if (!ctx->solid[n] && rs[n] > 0) {
        r.ux[n] = jx[n] / rs[n];
        r.uy[n] = jy[n] / rs[n];
      }
  }
  ctx->painted_C = false;
  ctx->paint_C.clear();
  ctx->paint_base_C.clear();
  ctx->rg = std::move(r);
  if (S.has_b) ctx->rb = S.b;
  return LB_OK;
}

}  // extern "C"
