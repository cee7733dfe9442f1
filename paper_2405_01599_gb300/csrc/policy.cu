// The numerical policy file of Sec. 2.3.2: "<keyword> = <value>" lines read
// by the meta-solvers before they run.  Host code only.
#include "common.cuh"

#include <cctype>
#include <cerrno>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>

namespace {

std::string trim(const std::string &s) {
    size_t a = 0, b = s.size();
    while (a < b && std::isspace((unsigned char)s[a])) a++;
    while (b > a && std::isspace((unsigned char)s[b - 1])) b--;
    return s.substr(a, b - a);
}

std::string upper(std::string s) {
    for (char &c : s) c = (char)std::toupper((unsigned char)c);
    return s;
}

// A real number; Fortran's exponent letter D is accepted as E.
bool parse_real(std::string v, double *out) {
    for (char &c : v)
        if (c == 'D' || c == 'd') c = 'E';
    if (v.empty()) return false;
    errno = 0;
    char *end = nullptr;
    const double x = std::strtod(v.c_str(), &end);
    if (errno != 0 || end == v.c_str() || *end != '\0') return false;
    *out = x;
    return true;
}

// Bytes, with an optional K / M / G / T suffix (powers of 1024) or a trailing B.
bool parse_bytes(std::string v, double *out) {
    v = upper(v);
    if (!v.empty() && v.back() == 'B') v.pop_back();
    double mult = 1.0;
    if (!v.empty()) {
        const char c = v.back();
        const double k = 1024.0;
        if (c == 'K') mult = k;
        else if (c == 'M') mult = k * k;
        else if (c == 'G') mult = k * k * k;
        else if (c == 'T') mult = k * k * k * k;
        if (mult != 1.0) v.pop_back();
    }
    double x = 0.0;
    if (!parse_real(trim(v), &x) || x < 0.0) return false;
    *out = x * mult;
    return true;
}

bool parse_int(const std::string &v, int32_t *out) {
    errno = 0;
    char *end = nullptr;
    const long x = std::strtol(v.c_str(), &end, 10);
    if (errno != 0 || end == v.c_str() || *end != '\0' || x < 0 || x > INT32_MAX) return false;
    *out = (int32_t)x;
    return true;
}

}  // namespace

extern "C" {

int xb_policy_parse(const char *text, xb_options *opt, int32_t *solver, double *max_memory,
                    int32_t *cpu) {
    if (!text || !opt) return xb::set_error(XB_EINVAL, "policy: NULL argument");
    int line_no = 0;
    const char *p = text;
    while (*p) {
        const char *e = std::strchr(p, '\n');
        std::string line = e ? std::string(p, e - p) : std::string(p);
        p = e ? e + 1 : p + line.size();
        line_no++;
        line = trim(line);
        if (line.empty() || line[0] == '#' || line[0] == '!') continue;
        const size_t eq = line.find('=');
        if (eq == std::string::npos)
            return xb::set_error(XB_EINVAL, "policy line %d: no '=' in \"%s\"", line_no,
                                 line.c_str());
        const std::string key = upper(trim(line.substr(0, eq)));
        const std::string val = trim(line.substr(eq + 1));
        const std::string uval = upper(val);
        bool ok = true;
        if (key == "POLICY") {
            // TIME is the default; a value the file does not register falls back to it
            opt->policy = uval == "ACCURACY" ? XB_POLICY_ACCURACY
                          : uval == "MEMORY" ? XB_POLICY_MEMORY
                          : uval == "STABLE" ? XB_POLICY_STABLE
                                             : XB_POLICY_TIME;
        } else if (key == "RESIDUAL") {
            double x = 0.0;
            ok = parse_real(val, &x) && x > 0.0;
            if (ok) opt->tol = x;
        } else if (key == "MAXTIME") {
            double x = 0.0;
            ok = parse_real(val, &x) && x > 0.0;
            if (ok) opt->maxtime_s = x;
        } else if (key == "PRECONDITIONER") {
            if (uval == "NONE" || uval == "NO") opt->precond = XB_PRECOND_NONE;
            else if (uval == "ILU0" || uval == "ILU(0)" || uval == "ILU")
                opt->precond = XB_PRECOND_ILU0;
            else ok = false;
        } else if (key == "SOLVER") {
            int32_t sv = -1;
            if (uval == "GMRES") sv = XB_SOLVER_GMRES;
            else if (uval == "BICGSTAB") sv = XB_SOLVER_BICGSTAB;
            else if (uval == "LANCZOS") sv = XB_SOLVER_LANCZOS;
            else if (uval == "ARNOLDI") sv = XB_SOLVER_ARNOLDI;
            ok = sv >= 0;
            if (ok && solver) *solver = sv;
        } else if (key == "MAXMEMORY") {
            double x = 0.0;
            ok = parse_bytes(val, &x);
            if (ok && max_memory) *max_memory = x;
        } else if (key == "CPU") {
            int32_t x = 0;
            ok = parse_int(val, &x);
            if (ok && cpu) *cpu = x;
        }  // other keywords: not registered, ignored
        if (!ok)
            return xb::set_error(XB_EINVAL, "policy line %d: bad value \"%s\" for %s", line_no,
                                 val.c_str(), key.c_str());
    }
    return XB_OK;
}

int xb_policy_read(const char *dir, int32_t id, xb_options *opt, int32_t *solver,
                   double *max_memory, int32_t *cpu) {
    if (!opt || id < 0) return xb::set_error(XB_EINVAL, "policy: bad argument");
    std::string path = dir && *dir ? std::string(dir) + "/" : std::string();
    path += "OPENATI_POLICY_INPUT." + std::to_string(id);
    FILE *f = std::fopen(path.c_str(), "rb");
    if (!f) return xb::set_error(XB_EINVAL, "policy: cannot open %s", path.c_str());
    std::string text;
    char buf[4096];
    size_t got;
    while ((got = std::fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, got);
    std::fclose(f);
    if (text.find('\0') != std::string::npos)
        return xb::set_error(XB_EINVAL, "policy: %s is not a text file", path.c_str());
    return xb_policy_parse(text.c_str(), opt, solver, max_memory, cpu);
}

}  // extern "C"
