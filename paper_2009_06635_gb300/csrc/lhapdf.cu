// lhapdf.cu -- reader of LHAPDF6 sets in the "lhagrid1" text format (host
// code only).  PDFFlow Sec. 2.2 loads the files of the LHAPDF directories
// directly, so a set needs no conversion; Sec. 2.3 takes the alpha_s nodes
// from the set's metadata.
//
// A set is a directory NAME/ holding NAME.info (YAML metadata) and one file
// per member, NAME_0000.dat, NAME_0001.dat, ...  What is read:
//   .info  Flavors: [pids], AlphaS_Qs: [Q nodes], AlphaS_Vals: [alpha_s]
//          (lists may span lines; other keys are ignored).
//   .dat   a YAML header ending with a line "---", then one block per Q
//          subgrid, each ended by "---":
//            line 1: the x knots;  line 2: the Q knots (GeV, not Q^2);
//            line 3: the flavour pids;
//            then nx * nq lines of nflav values xf, x the outer loop and Q
//            the inner one.
// Subgrids must share the x knots and the flavours (as LHAPDF sets do); the
// Q^2 knots are the squares of the Q knots, concatenated subgrid by subgrid,
// with the shared boundary knot repeated as pdf_grid_desc expects.
#include <cctype>
#include <cerrno>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "guard.cuh"
#include "pdf_internal.cuh"

using pdfgb::set_error;

struct pdf_lhapdf_set {
  std::vector<double> x, q2, values, as_q2, as_vals;
  std::vector<int> nq, pids;
};

namespace {

bool read_file(const char *path, std::string &text) {
  FILE *f = std::fopen(path, "rb");
  if (!f) return false;
  char buf[1 << 16];
  size_t k;
  text.clear();
  while ((k = std::fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, k);
  std::fclose(f);
  return true;
}

std::vector<std::string> split_lines(const std::string &t) {
  std::vector<std::string> lines;
  size_t a = 0;
  while (a <= t.size()) {
    size_t b = t.find('\n', a);
    if (b == std::string::npos) b = t.size();
    std::string l = t.substr(a, b - a);
    if (!l.empty() && l.back() == '\r') l.pop_back();
    lines.push_back(l);
    a = b + 1;
  }
  return lines;
}

std::string trim(const std::string &s) {
  size_t a = 0, b = s.size();
  while (a < b && std::isspace((unsigned char)s[a])) a++;
  while (b > a && std::isspace((unsigned char)s[b - 1])) b--;
  return s.substr(a, b - a);
}

// All numbers of a line (space or comma separated); false on a bad token.
bool numbers(const std::string &line, std::vector<double> &out) {
  out.clear();
  const char *p = line.c_str();
  while (*p) {
    while (*p && (std::isspace((unsigned char)*p) || *p == ',')) p++;
    if (!*p) break;
    char *end = nullptr;
    errno = 0;
    const double v = std::strtod(p, &end);
    if (end == p || errno == ERANGE) return false;
    out.push_back(v);
    p = end;
  }
  return true;
}

// The YAML list value of `key` in an .info text ("Key: [a, b, ...]", the
// list possibly continued on following lines); false if the key is absent.
bool info_list(const std::vector<std::string> &lines, const char *key, std::vector<double> &out, bool &bad) {
  const size_t kl = std::strlen(key);
  for (size_t i = 0; i < lines.size(); i++) {
    std::string l = lines[i];
    const size_t hash = l.find('#');
    if (hash != std::string::npos) l = l.substr(0, hash);
    l = trim(l);
    if (l.compare(0, kl, key) != 0 || l.size() <= kl || l[kl] != ':') continue;
    std::string v = trim(l.substr(kl + 1));
    while (v.find(']') == std::string::npos && i + 1 < lines.size()) v += " " + trim(lines[++i]);
    const size_t a = v.find('['), b = v.find(']');
    if (a == std::string::npos || b == std::string::npos || b < a) { bad = true; return true; }
    bad = !numbers(v.substr(a + 1, b - a - 1), out);
    return true;
  }
  return false;
}

bool is_sep(const std::string &l) { return trim(l) == "---"; }

int parse_dat(const char *path, pdf_lhapdf_set &S) {
  std::string text;
  if (!read_file(path, text)) return set_error(PDF_ERR_ARG, "lhapdf: cannot read %s", path);
  const std::vector<std::string> L = split_lines(text);
  size_t i = 0;
  while (i < L.size() && !is_sep(L[i])) i++;  // member header
  if (i == L.size()) return set_error(PDF_ERR_GRID, "lhapdf: %s: no '---' after the header", path);
  i++;
  std::vector<double> xs, qs, ps, row;
  int nblock = 0;
  while (true) {
    while (i < L.size() && trim(L[i]).empty()) i++;
    if (i >= L.size()) break;
    if (i + 2 >= L.size()) return set_error(PDF_ERR_GRID, "lhapdf: %s: truncated subgrid %d", path, nblock);
    if (!numbers(L[i], xs) || !numbers(L[i + 1], qs) || !numbers(L[i + 2], ps))
      return set_error(PDF_ERR_GRID, "lhapdf: %s: bad knot or flavour line in subgrid %d", path, nblock);
    i += 3;
    const size_t nx = xs.size(), nq = qs.size(), nf = ps.size();
    if (nx < 2 || nq < 2 || nf < 1)
      return set_error(PDF_ERR_GRID, "lhapdf: %s: subgrid %d has %zu x, %zu Q knots, %zu flavours", path, nblock,
                       nx, nq, nf);
    std::vector<int> pid(nf);
    for (size_t f = 0; f < nf; f++) {
      if (!(std::fabs(ps[f]) <= 1e6) || std::nearbyint(ps[f]) != ps[f])
        return set_error(PDF_ERR_GRID, "lhapdf: %s: flavour %g is not a particle id", path, ps[f]);
      pid[f] = (int)ps[f];
    }
    if (nblock == 0) {
      S.x = xs;
      S.pids = pid;
    } else {
      if (xs != S.x) return set_error(PDF_ERR_GRID, "lhapdf: %s: subgrid %d has different x knots", path, nblock);
      if (pid != S.pids) return set_error(PDF_ERR_GRID, "lhapdf: %s: subgrid %d has different flavours", path, nblock);
    }
    const size_t row0 = S.q2.size();
    for (double q : qs) S.q2.push_back(q * q);
    S.nq.push_back((int)nq);
    S.values.resize((row0 + nq) * nx * nf);
    for (size_t ix = 0; ix < nx; ix++)
      for (size_t iq = 0; iq < nq; iq++, i++) {
        if (i >= L.size() || !numbers(L[i], row) || row.size() != nf)
          return set_error(PDF_ERR_GRID, "lhapdf: %s: subgrid %d, value line for x %zu, Q %zu malformed", path,
                           nblock, ix, iq);
        double *dst = &S.values[((row0 + iq) * nx + ix) * nf];
        for (size_t f = 0; f < nf; f++) dst[f] = row[f];
      }
    if (i >= L.size() || !is_sep(L[i]))
      return set_error(PDF_ERR_GRID, "lhapdf: %s: subgrid %d not closed by '---'", path, nblock);
    i++;
    nblock++;
  }
  if (nblock == 0) return set_error(PDF_ERR_GRID, "lhapdf: %s: no subgrid", path);
  return PDF_OK;
}

int parse_info(const char *path, pdf_lhapdf_set &S) {
  std::string text;
  if (!read_file(path, text)) return set_error(PDF_ERR_ARG, "lhapdf: cannot read %s", path);
  const std::vector<std::string> L = split_lines(text);
  std::vector<double> fl, aq, av;
  bool bad = false;
  if (info_list(L, "Flavors", fl, bad)) {
    if (bad) return set_error(PDF_ERR_GRID, "lhapdf: %s: malformed Flavors", path);
    if (fl.size() != S.pids.size()) return set_error(PDF_ERR_GRID, "lhapdf: %s: Flavors disagree with the data", path);
    for (size_t f = 0; f < fl.size(); f++)
      if ((double)S.pids[f] != fl[f]) return set_error(PDF_ERR_GRID, "lhapdf: %s: Flavors disagree with the data", path);
  }
  const bool hq = info_list(L, "AlphaS_Qs", aq, bad);
  if (bad) return set_error(PDF_ERR_GRID, "lhapdf: %s: malformed AlphaS_Qs", path);
  const bool hv = info_list(L, "AlphaS_Vals", av, bad);
  if (bad) return set_error(PDF_ERR_GRID, "lhapdf: %s: malformed AlphaS_Vals", path);
  if (hq != hv || aq.size() != av.size())
    return set_error(PDF_ERR_GRID, "lhapdf: %s: AlphaS_Qs and AlphaS_Vals differ in length", path);
  S.as_q2.clear();
  for (double q : aq) S.as_q2.push_back(q * q);
  S.as_vals = av;
  return PDF_OK;
}

void fill_desc(const pdf_lhapdf_set &S, pdf_grid_desc *d) {
  std::memset(d, 0, sizeof *d);
  d->nx = (int)S.x.size();
  d->x_knots = S.x.data();
  d->nsub = (int)S.nq.size();
  d->nq = S.nq.data();
  d->q2_knots = S.q2.data();
  d->nflav = (int)S.pids.size();
  d->pids = S.pids.data();
  d->values = S.values.data();
  d->na = (int)S.as_q2.size();
  d->as_q2 = S.as_q2.empty() ? nullptr : S.as_q2.data();
  d->as_vals = S.as_vals.empty() ? nullptr : S.as_vals.data();
}

std::string member_path(const std::string &dir, const std::string &name, int m) {
  char buf[32];
  std::snprintf(buf, sizeof buf, "_%04d.dat", m);
  return dir + "/" + name + buf;
}

}  // namespace

extern "C" int pdf_lhapdf_read(const char *info_path, const char *dat_path, pdf_lhapdf_set **out) {
  if (!info_path || !dat_path || !out) return set_error(PDF_ERR_NULL, "pdf_lhapdf_read: NULL argument");
  *out = nullptr;
  return pdfgb::guarded("pdf_lhapdf_read", [&] {
    std::unique_ptr<pdf_lhapdf_set> S(new pdf_lhapdf_set());
    int rc = parse_dat(dat_path, *S);
    if (!rc) rc = parse_info(info_path, *S);
    if (!rc) *out = S.release();
    return rc;
  });
}

extern "C" int pdf_lhapdf_desc(const pdf_lhapdf_set *S, pdf_grid_desc *desc) {
  if (!S || !desc) return set_error(PDF_ERR_NULL, "pdf_lhapdf_desc: NULL argument");
  fill_desc(*S, desc);
  return PDF_OK;
}

extern "C" int pdf_lhapdf_free(pdf_lhapdf_set *S) {
  delete S;
  return PDF_OK;
}

namespace {

int load_lhapdf(const char *set_dir, int first_member, int nmem, pdf_grid **out) {
  std::string dir(set_dir);
  while (dir.size() > 1 && dir.back() == '/') dir.pop_back();
  const size_t slash = dir.find_last_of('/');
  const std::string name = slash == std::string::npos ? dir : dir.substr(slash + 1);
  const std::string info = dir + "/" + name + ".info";
  pdf_lhapdf_set *S0p = nullptr;
  int rc = pdf_lhapdf_read(info.c_str(), member_path(dir, name, first_member).c_str(), &S0p);
  if (rc) return rc;
  const std::unique_ptr<pdf_lhapdf_set> S0(S0p);
  pdf_grid_desc d;
  fill_desc(*S0, &d);
  if (nmem == 1) return pdf_load_grid(&d, out);
  std::vector<double> all;
  all.reserve(S0->values.size() * (size_t)nmem);
  all.insert(all.end(), S0->values.begin(), S0->values.end());
  for (int m = 1; m < nmem && !rc; m++) {
    pdf_lhapdf_set Sm;
    const std::string p = member_path(dir, name, first_member + m);
    rc = parse_dat(p.c_str(), Sm);
    if (!rc && (Sm.x != S0->x || Sm.q2 != S0->q2 || Sm.nq != S0->nq || Sm.pids != S0->pids))
      rc = set_error(PDF_ERR_GRID, "pdf_load_lhapdf: %s has other knots or flavours than member %d", p.c_str(),
                     first_member);
    if (!rc) all.insert(all.end(), Sm.values.begin(), Sm.values.end());
  }
  if (!rc) rc = pdf_load_grid_members(&d, nmem, all.data(), out);
  return rc;
}

}  // namespace

extern "C" int pdf_load_lhapdf(const char *set_dir, int first_member, int nmem, pdf_grid **out) {
  if (!set_dir || !out) return set_error(PDF_ERR_NULL, "pdf_load_lhapdf: NULL argument");
  *out = nullptr;
  if (first_member < 0 || nmem < 1 || nmem > 10000 - first_member)
    return set_error(PDF_ERR_ARG, "pdf_load_lhapdf: members %d..%lld outside 0..9999", first_member,
                     (long long)first_member + (nmem > 0 ? nmem - 1 : 0));
  return pdfgb::guarded("pdf_load_lhapdf", [&] { return load_lhapdf(set_dir, first_member, nmem, out); });
}
